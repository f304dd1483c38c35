// Macro solver for Eq. (homo) and direct simulation of Eq. (model).
//
// Macro step (HMM step 4): U_t = div(K grad U) in conservative flux form on
// the periodic N x N grid, face tensors K_f = (K_node + K_neighbour)/2, the
// mixed term by the 4-point average of cross differences (9-point stencil),
// Heun's RK2.  Every face flux is evaluated by both adjacent cells with the
// same operations, so sum(U) telescopes exactly apart from summation rounding.
//   N <= 64: one persistent CTA keeps U, U* and K in shared memory for all steps.
//   N  > 64: one launch per RK stage over the grid.
// The mass H^2 sum(U) of every step is summed in FP64.
//
// DNS: u_t = v1 D0x u + v2 D0y u + kappa (Dxx + Dyy) u, v = (-D0y psi, D0x psi),
// both RK stages fused per tile (u and psi staged with a halo of 2 in shared
// memory), one pass over HBM per time step: read u, read psi, write u.
#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "mlsd_internal.cuh"

namespace mlsd {
namespace {

// DIR = false: periodic in both directions.  DIR = true: the Sec. 4 set-up,
// Dirichlet in x1 -- column 0 is the boundary x1 = 0 (held by the caller) and
// the virtual column N the boundary x1 = 2 pi with value ur; the K field stays
// periodic (its column N is column 0).  Column 0 itself has no update (0).
template <typename real, bool DIR = false>
__device__ __forceinline__ real macro_rhs(int N, real invH, real inv4H, const real *U,
                                          const real *K11, const real *K12, const real *K22,
                                          int i, int j, real ur = (real)0)
{
    if (DIR && i == 0) return (real)0;
    const int ipk = (i + 1 == N) ? 0 : i + 1, im = (i == 0) ? N - 1 : i - 1;
    const int jp = (j + 1 == N) ? 0 : j + 1, jm = (j == 0) ? N - 1 : j - 1;
    const int c = j * N + i;
    const bool edge = DIR && i + 1 == N;        // east neighbours are the boundary value
    const real uE = edge ? ur : U[j * N + ipk], uEn = edge ? ur : U[jp * N + ipk];
    const real uEs = edge ? ur : U[jm * N + ipk];
    const real h = (real)0.5;
    // east face (i+1/2, j)
    real k11 = h * (K11[c] + K11[j * N + ipk]), k12 = h * (K12[c] + K12[j * N + ipk]);
    const real fe = k11 * (uE - U[c]) * invH
                  + k12 * (U[jp * N + i] + uEn - U[jm * N + i] - uEs) * inv4H;
    // west face (i-1/2, j)
    k11 = h * (K11[j * N + im] + K11[c]); k12 = h * (K12[j * N + im] + K12[c]);
    const real fw = k11 * (U[c] - U[j * N + im]) * invH
                  + k12 * (U[jp * N + im] + U[jp * N + i] - U[jm * N + im] - U[jm * N + i]) * inv4H;
    // north face (i, j+1/2)
    real k22 = h * (K22[c] + K22[jp * N + i]); k12 = h * (K12[c] + K12[jp * N + i]);
    const real fn = k22 * (U[jp * N + i] - U[c]) * invH
                  + k12 * (uE + uEn - U[j * N + im] - U[jp * N + im]) * inv4H;
    // south face (i, j-1/2)
    k22 = h * (K22[jm * N + i] + K22[c]); k12 = h * (K12[jm * N + i] + K12[c]);
    const real fs = k22 * (U[c] - U[jm * N + i]) * invH
                  + k12 * (uEs + uE - U[jm * N + im] - U[j * N + im]) * inv4H;
    return (fe - fw + fn - fs) * invH;
}

// deterministic FP64 block sum (all threads return the total)
__device__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

// one CTA, everything in shared memory (DIR: column 0 set to ul, east boundary ur)
template <typename real, bool DIR = false>
__global__ void __launch_bounds__(1024) k_macro_resident(int N, real *Ug, const double *Kg,
                                                         real dt, int nsteps, double *mass,
                                                         real ul = (real)0, real ur = (real)0)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real *U = reinterpret_cast<real *>(smem_raw);
    real *Us = U + N * N, *K11 = Us + N * N, *K12 = K11 + N * N, *K22 = K12 + N * N;
    __shared__ double red[32];
    const int NN = N * N;
    const double H = 2.0 * kPi / N;
    const real invH = (real)(1.0 / H), inv4H = (real)(1.0 / (4.0 * H));
    const double H2 = H * H;
    double m = 0.0;
    for (int c = threadIdx.x; c < NN; c += blockDim.x) {
        U[c] = (DIR && c % N == 0) ? ul : Ug[c];
        K11[c] = (real)Kg[3 * c]; K12[c] = (real)Kg[3 * c + 1]; K22[c] = (real)Kg[3 * c + 2];
        m += (double)U[c];
    }
    m = block_sum(m, red);
    if (threadIdx.x == 0 && mass) mass[0] = m * H2;
    for (int s = 1; s <= nsteps; ++s) {
        for (int c = threadIdx.x; c < NN; c += blockDim.x)
            Us[c] = U[c] + dt * macro_rhs<real, DIR>(N, invH, inv4H, U, K11, K12, K22, c % N, c / N, ur);
        __syncthreads();
        real nu[4];
        int k = 0;
        for (int c = threadIdx.x; c < NN; c += blockDim.x, ++k)
            nu[k] = (real)0.5 * (U[c] + Us[c] + dt * macro_rhs<real, DIR>(N, invH, inv4H, Us, K11, K12, K22, c % N, c / N, ur));
        __syncthreads();
        k = 0;
        m = 0.0;
        for (int c = threadIdx.x; c < NN; c += blockDim.x, ++k) { U[c] = nu[k]; m += (double)nu[k]; }
        if (mass) {
            m = block_sum(m, red);
            if (threadIdx.x == 0) mass[s] = m * H2;
        } else {
            __syncthreads();
        }
    }
    for (int c = threadIdx.x; c < NN; c += blockDim.x) Ug[c] = U[c];
}

template <typename real>
__global__ void k_split_K(int NN, const double *Kg, real *K11, real *K12, real *K22)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= NN) return;
    K11[c] = (real)Kg[3 * c]; K12[c] = (real)Kg[3 * c + 1]; K22[c] = (real)Kg[3 * c + 2];
}

// stage 1: Us = U + dt R(U); stage 2: U = (U + Us + dt R(Us)) / 2, with the block's
// share of sum(U) written to part[block]
template <typename real, bool SECOND, bool DIR = false>
__global__ void k_macro_stage(int N, real *U, real *Us, const real *K11, const real *K12,
                              const real *K22, real dt, double *part, real ur = (real)0)
{
    __shared__ double red[32];
    const int NN = N * N;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const double H = 2.0 * kPi / N;
    const real invH = (real)(1.0 / H), inv4H = (real)(1.0 / (4.0 * H));
    double m = 0.0;
    if (c < NN) {
        if (!SECOND) {
            Us[c] = U[c] + dt * macro_rhs<real, DIR>(N, invH, inv4H, U, K11, K12, K22, c % N, c / N, ur);
        } else {
            const real v = (real)0.5 * (U[c] + Us[c] + dt * macro_rhs<real, DIR>(N, invH, inv4H, Us, K11, K12, K22, c % N, c / N, ur));
            m = (double)v;
            // U is read by neighbours only in stage 1, so the in-place write is safe here
            U[c] = v;
        }
    }
    if (SECOND && part) {
        m = block_sum(m, red);
        if (threadIdx.x == 0) part[blockIdx.x] = m;
    }
}

// Dirichlet set-up: column 0 (the boundary x1 = 0) takes the boundary value
template <typename real>
__global__ void k_set_col0(int N, real *U, real ul)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < N) U[(long long)j * N] = ul;
}

template <typename real>
__global__ void k_mass_part(int NN, const real *U, double *part)
{
    __shared__ double red[32];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    double m = c < NN ? (double)U[c] : 0.0;
    m = block_sum(m, red);
    if (threadIdx.x == 0) part[blockIdx.x] = m;
}

// mass[s] = H^2 * sum_b part[s][b]
__global__ void k_mass_final(int nsteps1, int nblocks, const double *part, double H2, double *mass)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsteps1) return;
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += part[(long long)s * nblocks + b];
    mass[s] = t * H2;
}

__global__ void k_kmax(int NN, const double *K, double *out)
{
    __shared__ double red[32];
    double m = 0.0;
    for (int c = threadIdx.x; c < NN; c += blockDim.x)
        m = fmax(m, K[3 * c] + K[3 * c + 2] + fabs(K[3 * c + 1]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
        *out = t;
    }
}

// ---------------------------------------------------------------------------
// DNS step, both Heun stages fused, one pass over HBM (read u, read psi,
// write u).  A CTA owns a 128 x 64 output tile.  u and psi are staged with a
// 2-row / 8-column halo by 16-byte cp.async copies.  Thread (g, seg) owns the
// 4 columns x0 - 4 + 4g .. +3 (g = 0 and 33 are halo groups) and the 8 output
// rows y0 + 8 seg .. +7: it computes stage 1 on those rows plus one row above
// and below (kept in registers), publishes its left and right edge columns of
// the stage-1 field for its own rows, and after one barrier computes stage 2
// on its output rows from registers (north, south) and the neighbours' edges
// (east, west).
constexpr int DTX = 128, DRS = 8;
constexpr int DG = DTX / 4 + 2;                // column groups incl. the two halo groups
constexpr int DLX = DTX + 16;                  // staged columns x0-8 .. x0+TX+7
template <int DTY> struct DnsTile {
    static constexpr int DSEG = DTY / DRS;     // row segments
    static constexpr int DTH = DG * DSEG;      // threads
    static constexpr int DLY = DTY + 4;        // staged rows y0-2 .. y0+TY+1
    static constexpr size_t SMEM = (size_t)2 * DLY * DLX * 4 + (size_t)2 * DTY * DG * 4;
};

__device__ __forceinline__ void cp16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::
                 "r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}

template <int DTY>
__global__ void __launch_bounds__(DnsTile<DTY>::DTH) k_dns_step(int nf, const float *__restrict__ u,
                                                               const float *__restrict__ psi,
                                                               float *__restrict__ un, float ax,
                                                               float kd, float dt)
{
    constexpr int DLY = DnsTile<DTY>::DLY, DTH = DnsTile<DTY>::DTH;
    extern __shared__ __align__(16) float dsm[];
    float *su = dsm;                          // [DLY][DLX]
    float *sp = su + DLY * DLX;               // [DLY][DLX]
    float *eL = sp + DLY * DLX;               // [DTY][DG]  stage-1 value of a group's column 0
    float *eR = eL + DTY * DG;                // [DTY][DG]  ... of its column 3
    const int x0 = blockIdx.x * DTX, y0 = blockIdx.y * DTY;
    for (int k = threadIdx.x; k < DLY * (DLX / 4); k += DTH) {
        const int r = k / (DLX / 4), q = k % (DLX / 4);
        int gy = y0 - 2 + r; gy = gy < 0 ? gy + nf : (gy >= nf ? gy - nf : gy);
        int gx = x0 - 8 + 4 * q; gx = gx < 0 ? gx + nf : (gx >= nf ? gx - nf : gx);
        const long long off = (long long)gy * nf + gx;
        cp16(su + r * DLX + 4 * q, u + off);
        cp16(sp + r * DLX + 4 * q, psi + off);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();

    const int g = threadIdx.x % DG, seg = threadIdx.x / DG;
    const int c0 = 4 + 4 * g;                 // staged column of the group's first column
    // the last warp is partial (DTH = 34 DTY/8 threads): shuffles name its lanes only;
    // its last thread is a g = DG - 1 thread, so no lane reads past it
    const int lane = threadIdx.x & 31, wbase = threadIdx.x & ~31;
    const unsigned wmask = DTH - wbase >= 32 ? 0xffffffffu : ((1u << (DTH - wbase)) - 1u);
    const bool edgeW = g == 0 || lane == 0, edgeE = g == DG - 1 || lane == 31;
    // x + dt f(x) = x + cD (xE + xW + xN + xS - 4 x)
    //                 + cA [(psiS - psiN)(xE - xW) + (psiE - psiW)(xN - xS)],
    // cA = dt / (4 h^2), cD = dt kappa / h^2; the Laplacian stays a difference so
    // that rounding does not bias the sum of u
    const float cA = dt * ax * ax, cD = dt * kd;
    const int rbase = 2 + DRS * seg;          // staged row of the segment's first output row
    // ---- stage 1 on rows rbase-1 .. rbase+DRS (registers s[0..DRS+1]) ----
    float s1[DRS + 2][4];
    {
        float um[4], uc[4], up[4], pm[4], pc[4], pp[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            um[c] = su[(rbase - 2) * DLX + c0 + c]; uc[c] = su[(rbase - 1) * DLX + c0 + c];
            pm[c] = sp[(rbase - 2) * DLX + c0 + c]; pc[c] = sp[(rbase - 1) * DLX + c0 + c];
        }
#pragma unroll
        for (int k = 0; k < DRS + 2; ++k) {
            const int r = rbase - 1 + k;
            const float4 un4 = *reinterpret_cast<const float4 *>(su + (r + 1) * DLX + c0);
            const float4 pn4 = *reinterpret_cast<const float4 *>(sp + (r + 1) * DLX + c0);
            up[0] = un4.x; up[1] = un4.y; up[2] = un4.z; up[3] = un4.w;
            pp[0] = pn4.x; pp[1] = pn4.y; pp[2] = pn4.z; pp[3] = pn4.w;
            // the neighbouring columns come from the neighbouring lanes (the groups of a
            // segment are consecutive threads); lanes at a warp or segment edge read
            // shared memory (a scalar column read is a 4-way bank conflict)
            float uw = __shfl_up_sync(wmask, uc[3], 1), ue = __shfl_down_sync(wmask, uc[0], 1);
            float pw = __shfl_up_sync(wmask, pc[3], 1), pe = __shfl_down_sync(wmask, pc[0], 1);
            if (edgeW) { uw = su[r * DLX + c0 - 1]; pw = sp[r * DLX + c0 - 1]; }
            if (edgeE) { ue = su[r * DLX + c0 + 4]; pe = sp[r * DLX + c0 + 4]; }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float uE = c < 3 ? uc[c + 1] : ue, uW = c > 0 ? uc[c - 1] : uw;
                const float pE = c < 3 ? pc[c + 1] : pe, pW = c > 0 ? pc[c - 1] : pw;
                float t = (pm[c] - pp[c]) * (uE - uW);
                t = fmaf(pE - pW, up[c] - um[c], t);
                const float lap = fmaf(-4.0f, uc[c], (uE + uW) + (up[c] + um[c]));
                s1[k][c] = fmaf(cA, t, fmaf(cD, lap, uc[c]));
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) { um[c] = uc[c]; uc[c] = up[c]; pm[c] = pc[c]; pc[c] = pp[c]; }
        }
    }
    // publish the edge columns of the stage-1 field on the segment's own rows
#pragma unroll
    for (int k = 0; k < DRS; ++k) {
        eL[(DRS * seg + k) * DG + g] = s1[k + 1][0];
        eR[(DRS * seg + k) * DG + g] = s1[k + 1][3];
    }
    __syncthreads();
    if (g == 0 || g == DG - 1) return;        // halo groups: stage-1 values only
    // ---- stage 2 on the output rows ----
    {
        float pm[4], pc[4], pp[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            pm[c] = sp[(rbase - 1) * DLX + c0 + c];
            pc[c] = sp[rbase * DLX + c0 + c];
        }
        const int gx = x0 + 4 * (g - 1);
#pragma unroll
        for (int k = 0; k < DRS; ++k) {
            const int r = rbase + k;
            const float4 pn4 = *reinterpret_cast<const float4 *>(sp + (r + 1) * DLX + c0);
            pp[0] = pn4.x; pp[1] = pn4.y; pp[2] = pn4.z; pp[3] = pn4.w;
            const float pw = sp[r * DLX + c0 - 1], pe = sp[r * DLX + c0 + 4];
            const float sw = eR[(DRS * seg + k) * DG + g - 1], se = eL[(DRS * seg + k) * DG + g + 1];
            const float4 u4 = *reinterpret_cast<const float4 *>(su + r * DLX + c0);
            const float uo[4] = {u4.x, u4.y, u4.z, u4.w};
            float o[4];
            // (u + s + dt f(s)) / 2
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float sC = s1[k + 1][c], sN = s1[k + 2][c], sS = s1[k][c];
                const float sE = c < 3 ? s1[k + 1][c + 1] : se, sW = c > 0 ? s1[k + 1][c - 1] : sw;
                const float pE = c < 3 ? pc[c + 1] : pe, pW = c > 0 ? pc[c - 1] : pw;
                float t = (pm[c] - pp[c]) * (sE - sW);
                t = fmaf(pE - pW, sN - sS, t);
                const float lap = fmaf(-4.0f, sC, (sE + sW) + (sN + sS));
                o[c] = 0.5f * (uo[c] + fmaf(cA, t, fmaf(cD, lap, sC)));
            }
            *reinterpret_cast<float4 *>(un + (long long)(y0 + DRS * seg + k) * nf + gx) =
                make_float4(o[0], o[1], o[2], o[3]);
#pragma unroll
            for (int c = 0; c < 4; ++c) { pm[c] = pc[c]; pc[c] = pp[c]; }
        }
    }
}

// DNS with the Sec. 4 boundaries (Dirichlet in x1, periodic in x2): one launch
// per Heun stage, one thread per node.  Column 0 is the boundary x1 = 0 (held
// at ul), the virtual column nf the boundary x1 = 2 pi (value ur); psi and the
// velocity stay periodic.  Stage 1: s = u + dt f(u) into `out`; stage 2:
// out = (u + s + dt f(s)) / 2 with `s` the stage-1 field.  The same folded
// constants as k_dns_step: cA = dt / (4 h^2) on psi differences times u
// differences, cD = dt kappa / h^2 on the Laplacian (kept as a difference).
template <bool SECOND, typename real>
__global__ void k_dns_dir_stage(int nf, const real *__restrict__ u, const real *__restrict__ sfield,
                                const float *__restrict__ psi, real *__restrict__ out, real cA,
                                real cD, real ul, real ur)
{
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= (long long)nf * nf) return;
    const int a = (int)(c % nf), b = (int)(c / nf);
    if (a == 0) { out[c] = ul; return; }
    const real *x = SECOND ? sfield : u;
    const int bp = b + 1 == nf ? 0 : b + 1, bm = b == 0 ? nf - 1 : b - 1;
    const int ap = a + 1 == nf ? 0 : a + 1;
    const long long row = (long long)b * nf;
    const real xc = x[c];
    const real xE = a + 1 == nf ? ur : x[row + ap], xW = x[c - 1];
    const real xN = x[(long long)bp * nf + a], xS = x[(long long)bm * nf + a];
    // dt (v1 D0x + v2 D0y) x = cA [(psiS - psiN)(xE - xW) + (psiE - psiW)(xN - xS)]
    const real pN = psi[(long long)bp * nf + a], pS = psi[(long long)bm * nf + a];
    const real pE = psi[row + ap], pW = psi[row + a - 1];
    real t = (pS - pN) * (xE - xW);
    t = fma(pE - pW, xN - xS, t);
    const real lap = fma((real)-4, xc, (xE + xW) + (xN + xS));
    const real g = fma(cA, t, fma(cD, lap, xc));
    out[c] = SECOND ? (real)0.5 * (u[c] + g) : g;
}

// max over the grid of |v1| + |v2| (non-negative floats order like their bit patterns)
__global__ void k_dns_vmax(int nf, const float *psi, float ax, unsigned *out)
{
    float m = 0.f;
    const long long n2 = (long long)nf * nf;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n2;
         c += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(c / nf), a = (int)(c % nf);
        const int bp = b + 1 == nf ? 0 : b + 1, bm = b == 0 ? nf - 1 : b - 1;
        const int ap = a + 1 == nf ? 0 : a + 1, am = a == 0 ? nf - 1 : a - 1;
        const float v1 = (psi[(long long)bm * nf + a] - psi[(long long)bp * nf + a]) * ax;
        const float v2 = (psi[(long long)b * nf + ap] - psi[(long long)b * nf + am]) * ax;
        m = fmaxf(m, fabsf(v1) + fabsf(v2));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// box average onto the macro grid; box[j*N+i] = FP64 sum of the box
__global__ void k_coarse(int nf, const float *u, int N, float *U, double *box)
{
    __shared__ double red[32];
    const int i = blockIdx.x, j = blockIdx.y, r = nf / N;
    double s = 0.0;
    for (int k = threadIdx.x; k < r * r; k += blockDim.x) {
        const int db = k / r, da = k % r;
        int b = j * r - r / 2 + db; b = b < 0 ? b + nf : (b >= nf ? b - nf : b);
        int a = i * r - r / 2 + da; a = a < 0 ? a + nf : (a >= nf ? a - nf : a);
        s += (double)u[(long long)b * nf + a];
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        U[j * N + i] = (float)(s / ((double)r * r));
        if (box) box[j * N + i] = s;
    }
}

__global__ void k_sum(int n, const double *x, double scale, double *out)
{
    __shared__ double red[32];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += x[k];
    s = block_sum(s, red);
    if (threadIdx.x == 0) *out = s * scale;
}

}  // namespace

size_t macro_scratch_bytes(int N, int precision, int nsteps)
{
    const size_t rs = precision == MLSD_FP64 ? 8 : 4;
    const size_t NN = (size_t)N * N;
    if (N <= 64) return 0;
    const size_t nblocks = (NN + 255) / 256;
    return 4 * NN * rs + 256 + (size_t)(nsteps + 1) * nblocks * sizeof(double);
}

template <typename real, bool DIR>
static cudaError_t macro_run_t(int N, real *U, const double *K, double dt, int nsteps,
                               double *mass, void *scratch, cudaStream_t s, double ul, double ur)
{
    const int NN = N * N;
    const double H = 2.0 * kPi / N;
    if (N <= 64) {
        const size_t smem = 5 * (size_t)NN * sizeof(real);
        cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(&k_macro_resident<real, DIR>),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const int threads = NN >= 1024 ? 1024 : ((NN + 31) / 32) * 32;
        count_launches(1);
        k_macro_resident<real, DIR><<<1, threads, smem, s>>>(N, U, K, (real)dt, nsteps, mass,
                                                             (real)ul, (real)ur);
        return cudaGetLastError();
    }
    real *Us = static_cast<real *>(scratch);
    real *K11 = Us + NN, *K12 = K11 + NN, *K22 = K12 + NN;
    const int th = 256, nb = (NN + th - 1) / th;
    double *part = reinterpret_cast<double *>(
        (reinterpret_cast<uintptr_t>(K22 + NN) + 255) & ~(uintptr_t)255);
    count_launches(1 + 2 * (long long)nsteps + (mass ? 2 : 0) + (DIR ? 1 : 0));
    k_split_K<real><<<nb, th, 0, s>>>(NN, K, K11, K12, K22);
    if (DIR) k_set_col0<real><<<(N + 255) / 256, 256, 0, s>>>(N, U, (real)ul);
    if (mass) k_mass_part<real><<<nb, th, 0, s>>>(NN, U, part);
    for (int st = 1; st <= nsteps; ++st) {
        k_macro_stage<real, false, DIR><<<nb, th, 0, s>>>(N, U, Us, K11, K12, K22, (real)dt, nullptr,
                                                          (real)ur);
        k_macro_stage<real, true, DIR><<<nb, th, 0, s>>>(N, U, Us, K11, K12, K22, (real)dt,
                                                         mass ? part + (size_t)st * nb : nullptr,
                                                         (real)ur);
    }
    if (mass) k_mass_final<<<(nsteps + 1 + 127) / 128, 128, 0, s>>>(nsteps + 1, nb, part, H * H, mass);
    return cudaGetLastError();
}

cudaError_t macro_run(int N, void *U, int precision, const double *K, double dt, int nsteps,
                      double *mass_dev, void *scratch, cudaStream_t s)
{
    if (precision == MLSD_FP64)
        return macro_run_t<double, false>(N, static_cast<double *>(U), K, dt, nsteps, mass_dev,
                                          scratch, s, 0.0, 0.0);
    return macro_run_t<float, false>(N, static_cast<float *>(U), K, dt, nsteps, mass_dev, scratch,
                                     s, 0.0, 0.0);
}

cudaError_t macro_run_dirichlet(int N, void *U, int precision, const double *K, double dt,
                                int nsteps, double ul, double ur, double *mass_dev, void *scratch,
                                cudaStream_t s)
{
    if (precision == MLSD_FP64)
        return macro_run_t<double, true>(N, static_cast<double *>(U), K, dt, nsteps, mass_dev,
                                         scratch, s, ul, ur);
    return macro_run_t<float, true>(N, static_cast<float *>(U), K, dt, nsteps, mass_dev, scratch,
                                    s, ul, ur);
}

cudaError_t macro_dt_max(int N, const double *K, double *max_dev, cudaStream_t s)
{
    count_launches(1);
    k_kmax<<<1, 1024, 0, s>>>(N * N, K, max_dev);
    return cudaGetLastError();
}

template <int DTY>
static cudaError_t dns_launch(int nf, const float *a, const float *psi, float *b, float ax, float kd,
                              float dt, cudaStream_t s)
{
    using T = DnsTile<DTY>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(&k_dns_step<DTY>),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_dns_step<DTY><<<dim3(nf / DTX, nf / DTY), T::DTH, T::SMEM, s>>>(nf, a, psi, b, ax, kd, dt);
    return cudaGetLastError();
}

// tile height: 64 rows (2 CTAs/SM) or 32 rows (4 CTAs/SM, loads of one CTA overlap
// another's compute); picked once per process by timing both on the caller's grid
static int g_dns_ty = 0;

cudaError_t dns_run(int nf, float *u, float *u_tmp, const float *psi, double kappa, double dt,
                    int nsteps, cudaStream_t s)
{
    const double h = 2.0 * kPi / nf;
    const float ax = (float)(1.0 / (2.0 * h));
    const float kd = (float)(kappa / (h * h));
    if (const char *env = std::getenv("MLSD_DNS_TY")) g_dns_ty = std::atoi(env) == 32 ? 32 : 64;
    if (g_dns_ty == 0 && nsteps > 0) {
        // one trial step of each into u_tmp (u is not modified), best of two
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        for (int ty : {64, 32}) {
            float t = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, s);
                cudaError_t e = ty == 64 ? dns_launch<64>(nf, u, psi, u_tmp, ax, kd, (float)dt, s)
                                         : dns_launch<32>(nf, u, psi, u_tmp, ax, kd, (float)dt, s);
                cudaEventRecord(e1, s);
                if (e != cudaSuccess) return e;
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) t = std::min(t, ms);
            }
            count_launches(3);
            if (t < best) { best = t; g_dns_ty = ty; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    float *a = u, *b = u_tmp;
    count_launches(nsteps);
    for (int st = 0; st < nsteps; ++st) {
        cudaError_t e = g_dns_ty == 32 ? dns_launch<32>(nf, a, psi, b, ax, kd, (float)dt, s)
                                       : dns_launch<64>(nf, a, psi, b, ax, kd, (float)dt, s);
        if (e != cudaSuccess) return e;
        float *t = a; a = b; b = t;
    }
    if (a != u)
        return cudaMemcpyAsync(u, a, (size_t)nf * nf * sizeof(float), cudaMemcpyDeviceToDevice, s);
    return cudaGetLastError();
}

template <typename real>
static cudaError_t dns_run_dirichlet_t(int nf, real *u, real *u_tmp, const float *psi,
                                       double kappa, double dt, int nsteps, double ul, double ur,
                                       cudaStream_t s)
{
    const double h = 2.0 * kPi / nf;
    const real cA = (real)(dt / (4.0 * h * h));
    const real cD = (real)(dt * kappa / (h * h));
    const long long n2 = (long long)nf * nf;
    const unsigned nb = (unsigned)((n2 + 255) / 256);
    count_launches(1 + 2 * (long long)nsteps);
    k_set_col0<real><<<(nf + 255) / 256, 256, 0, s>>>(nf, u, (real)ul);
    for (int st = 0; st < nsteps; ++st) {
        k_dns_dir_stage<false, real><<<nb, 256, 0, s>>>(nf, u, nullptr, psi, u_tmp, cA, cD,
                                                        (real)ul, (real)ur);
        // stage 2 writes u in place: each node reads only its own u
        k_dns_dir_stage<true, real><<<nb, 256, 0, s>>>(nf, u, u_tmp, psi, u, cA, cD, (real)ul,
                                                       (real)ur);
    }
    return cudaGetLastError();
}

cudaError_t dns_run_dirichlet(int nf, void *u, void *u_tmp, const float *psi, int precision,
                              double kappa, double dt, int nsteps, double ul, double ur,
                              cudaStream_t s)
{
    if (precision == MLSD_FP64)
        return dns_run_dirichlet_t<double>(nf, static_cast<double *>(u), static_cast<double *>(u_tmp),
                                           psi, kappa, dt, nsteps, ul, ur, s);
    return dns_run_dirichlet_t<float>(nf, static_cast<float *>(u), static_cast<float *>(u_tmp), psi,
                                      kappa, dt, nsteps, ul, ur, s);
}

cudaError_t dns_vmax(int nf, const float *psi, unsigned *vmax_bits, cudaStream_t s)
{
    const double h = 2.0 * kPi / nf;
    cudaError_t e = cudaMemsetAsync(vmax_bits, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_dns_vmax<<<1024, 256, 0, s>>>(nf, psi, (float)(1.0 / (2.0 * h)), vmax_bits);
    return cudaGetLastError();
}

cudaError_t coarse_grain(int nf, const float *u, int N, float *U, double *mass_dev,
                         cudaStream_t s)
{
    double *box = mass_dev ? mass_dev + 1 : nullptr;
    count_launches(mass_dev ? 2 : 1);
    k_coarse<<<dim3(N, N), 256, 0, s>>>(nf, u, N, U, box);
    if (mass_dev) {
        const double h = 2.0 * kPi / nf;
        k_sum<<<1, 1024, 0, s>>>(N * N, box, h * h, mass_dev);
    }
    return cudaGetLastError();
}

}  // namespace mlsd

// ---------------------------------------------------------------------------
// Coarse-graining without allocation.
//
// Callers that must not allocate device memory (code running inside a host
// callback or a memory-pool-free embedding, allocator-less runtimes, or code
// that has handed all device memory to its own pool) get a variant of
// mlsd_coarse_grain whose scratch -- the FP64 box sums and the mass -- lives
// in the file-scope array below.  It holds 1 + MLSD_NOALLOC_MAX_MACRO^2
// doubles (about 512 KiB) on every device that loads the library, until the
// process exits.  Host code may not use the array's name as a pointer (it is
// a host-side stand-in): its device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call there.
namespace mlsd {
namespace {
constexpr int kNoallocMax = MLSD_NOALLOC_MAX_MACRO;
constexpr int kNoallocDevices = 64;
static __device__ __align__(256) double g_cg_scratch[1 + kNoallocMax * kNoallocMax];
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kNoallocDevices] = {};

cudaError_t noalloc_scratch(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoallocDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_cg_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}
}  // namespace
}  // namespace mlsd

extern "C" int mlsd_coarse_grain_noalloc(int nf, const float *u_dev, int n_macro, float *U_dev,
                                         double *mass_out_host, void *cuda_stream)
{
    using namespace mlsd;
    if (nf < 1 || n_macro < 1 || nf % n_macro || !u_dev || !U_dev) return MLSD_EINVAL;
    if (n_macro > kNoallocMax) return MLSD_EINVAL;          // scratch holds N <= 256 only
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    double *scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess) return MLSD_ECUDA;
    // every box sum and the mass are overwritten by this call: nothing carries over
    cudaError_t e = coarse_grain(nf, u_dev, n_macro, U_dev, mass_out_host ? scratch : nullptr, s);
    if (e == cudaSuccess && mass_out_host)
        e = cudaMemcpyAsync(mass_out_host, scratch, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && mass_out_host) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? MLSD_OK : MLSD_ECUDA;
}
