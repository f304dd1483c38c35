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
#include <string>
#include <vector>

#include <cuda.h>

#include "async_copy.cuh"
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

// Both Heun stages of one tile from its staged u and psi (rows y0-2 .. y0+DTY+1,
// columns x0-8 .. x0+DTX+7 in su, sp): stage 1 in registers, the edge columns
// of the stage-1 field through eL / eR and one CTA barrier, stage 2 stored to un.
template <int DTY>
__device__ __forceinline__ void dns_tile(const float *su, const float *sp, float *eL, float *eR,
                                         int nf, int x0, int y0, float *__restrict__ un, float ax,
                                         float kd, float dt)
{
    constexpr int DTH = DnsTile<DTY>::DTH;
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
    // ---- stage 2 on the output rows (the halo groups hold stage-1 values only) ----
    if (g != 0 && g != DG - 1) {
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

// f32x2 helpers: a - b as fma(b, -1, a), which rounds like the subtraction
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 bcast2(float v) { return make_float2(v, v); }

// dns_tile with the columns of a thread's group in f32x2 pairs (0, 1) and (2, 3):
// every stencil operation is one FFMA2 / FADD2 / FMUL2 for two cells, with the
// same operands and order per cell as dns_tile, so the result is the same bit
// for bit.  The neighbour pairs that straddle the two halves, (1, 2), (w, 0) and
// (3, e), are assembled from registers.
template <int DTY>
__device__ __forceinline__ void dns_tile2(const float *su, const float *sp, float *eL, float *eR,
                                          int nf, int x0, int y0, float *__restrict__ un, float ax,
                                          float kd, float dt)
{
    constexpr int DTH = DnsTile<DTY>::DTH;
    const int g = threadIdx.x % DG, seg = threadIdx.x / DG;
    const int c0 = 4 + 4 * g;
    const int lane = threadIdx.x & 31, wbase = threadIdx.x & ~31;
    const unsigned wmask = DTH - wbase >= 32 ? 0xffffffffu : ((1u << (DTH - wbase)) - 1u);
    const bool edgeW = g == 0 || lane == 0, edgeE = g == DG - 1 || lane == 31;
    const float2 cA = bcast2(dt * ax * ax), cD = bcast2(dt * kd), m4 = bcast2(-4.0f);
    const int rbase = 2 + DRS * seg;
    float2 sA[DRS + 2], sB[DRS + 2];             // stage-1 field, columns (0, 1) and (2, 3)
    {
        auto ld2 = [&](const float *base, int r, float2 &a, float2 &b) {
            const float4 v = *reinterpret_cast<const float4 *>(base + r * DLX + c0);
            a = make_float2(v.x, v.y);
            b = make_float2(v.z, v.w);
        };
        float2 umA, umB, ucA, ucB, pmA, pmB, pcA, pcB;
        ld2(su, rbase - 2, umA, umB); ld2(su, rbase - 1, ucA, ucB);
        ld2(sp, rbase - 2, pmA, pmB); ld2(sp, rbase - 1, pcA, pcB);
#pragma unroll
        for (int k = 0; k < DRS + 2; ++k) {
            const int r = rbase - 1 + k;
            float2 upA, upB, ppA, ppB;
            ld2(su, r + 1, upA, upB);
            ld2(sp, r + 1, ppA, ppB);
            float uw = __shfl_up_sync(wmask, ucB.y, 1), ue = __shfl_down_sync(wmask, ucA.x, 1);
            float pw = __shfl_up_sync(wmask, pcB.y, 1), pe = __shfl_down_sync(wmask, pcA.x, 1);
            if (edgeW) { uw = su[r * DLX + c0 - 1]; pw = sp[r * DLX + c0 - 1]; }
            if (edgeE) { ue = su[r * DLX + c0 + 4]; pe = sp[r * DLX + c0 + 4]; }
            const float2 uMid = make_float2(ucA.y, ucB.x), pMid = make_float2(pcA.y, pcB.x);
            const float2 uWA = make_float2(uw, ucA.x), uEB = make_float2(ucB.y, ue);
            const float2 pWA = make_float2(pw, pcA.x), pEB = make_float2(pcB.y, pe);
            {   // columns 0, 1: east (1, 2), west (w, 0)
                float2 t = __fmul2_rn(sub2(pmA, ppA), sub2(uMid, uWA));
                t = __ffma2_rn(sub2(pMid, pWA), sub2(upA, umA), t);
                const float2 lap = __ffma2_rn(m4, ucA, __fadd2_rn(__fadd2_rn(uMid, uWA),
                                                                 __fadd2_rn(upA, umA)));
                sA[k] = __ffma2_rn(cA, t, __ffma2_rn(cD, lap, ucA));
            }
            {   // columns 2, 3: east (3, e), west (1, 2)
                float2 t = __fmul2_rn(sub2(pmB, ppB), sub2(uEB, uMid));
                t = __ffma2_rn(sub2(pEB, pMid), sub2(upB, umB), t);
                const float2 lap = __ffma2_rn(m4, ucB, __fadd2_rn(__fadd2_rn(uEB, uMid),
                                                                 __fadd2_rn(upB, umB)));
                sB[k] = __ffma2_rn(cA, t, __ffma2_rn(cD, lap, ucB));
            }
            umA = ucA; umB = ucB; ucA = upA; ucB = upB;
            pmA = pcA; pmB = pcB; pcA = ppA; pcB = ppB;
        }
    }
#pragma unroll
    for (int k = 0; k < DRS; ++k) {
        eL[(DRS * seg + k) * DG + g] = sA[k + 1].x;
        eR[(DRS * seg + k) * DG + g] = sB[k + 1].y;
    }
    __syncthreads();
    if (g != 0 && g != DG - 1) {
        const float4 pm4 = *reinterpret_cast<const float4 *>(sp + (rbase - 1) * DLX + c0);
        const float4 pc4 = *reinterpret_cast<const float4 *>(sp + rbase * DLX + c0);
        float2 pmA = make_float2(pm4.x, pm4.y), pmB = make_float2(pm4.z, pm4.w);
        float2 pcA = make_float2(pc4.x, pc4.y), pcB = make_float2(pc4.z, pc4.w);
        const int gx = x0 + 4 * (g - 1);
        const float2 half = bcast2(0.5f);
#pragma unroll
        for (int k = 0; k < DRS; ++k) {
            const int r = rbase + k;
            const float4 pn4 = *reinterpret_cast<const float4 *>(sp + (r + 1) * DLX + c0);
            const float2 ppA = make_float2(pn4.x, pn4.y), ppB = make_float2(pn4.z, pn4.w);
            const float pw = sp[r * DLX + c0 - 1], pe = sp[r * DLX + c0 + 4];
            const float sw = eR[(DRS * seg + k) * DG + g - 1], se = eL[(DRS * seg + k) * DG + g + 1];
            const float4 u4 = *reinterpret_cast<const float4 *>(su + r * DLX + c0);
            const float2 uoA = make_float2(u4.x, u4.y), uoB = make_float2(u4.z, u4.w);
            const float2 sCA = sA[k + 1], sCB = sB[k + 1];
            const float2 sMid = make_float2(sCA.y, sCB.x), pMid = make_float2(pcA.y, pcB.x);
            const float2 sWA = make_float2(sw, sCA.x), sEB = make_float2(sCB.y, se);
            const float2 pWA = make_float2(pw, pcA.x), pEB = make_float2(pcB.y, pe);
            float2 oA, oB;
            {
                float2 t = __fmul2_rn(sub2(pmA, ppA), sub2(sMid, sWA));
                t = __ffma2_rn(sub2(pMid, pWA), sub2(sA[k + 2], sA[k]), t);
                const float2 lap = __ffma2_rn(m4, sCA, __fadd2_rn(__fadd2_rn(sMid, sWA),
                                                                 __fadd2_rn(sA[k + 2], sA[k])));
                oA = __fmul2_rn(half, __fadd2_rn(uoA, __ffma2_rn(cA, t, __ffma2_rn(cD, lap, sCA))));
            }
            {
                float2 t = __fmul2_rn(sub2(pmB, ppB), sub2(sEB, sMid));
                t = __ffma2_rn(sub2(pEB, pMid), sub2(sB[k + 2], sB[k]), t);
                const float2 lap = __ffma2_rn(m4, sCB, __fadd2_rn(__fadd2_rn(sEB, sMid),
                                                                 __fadd2_rn(sB[k + 2], sB[k])));
                oB = __fmul2_rn(half, __fadd2_rn(uoB, __ffma2_rn(cA, t, __ffma2_rn(cD, lap, sCB))));
            }
            *reinterpret_cast<float4 *>(un + (long long)(y0 + DRS * seg + k) * nf + gx) =
                make_float4(oA.x, oA.y, oB.x, oB.y);
            pmA = pcA; pmB = pcB; pcA = ppA; pcB = ppB;
        }
    }
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
    dns_tile<DTY>(su, sp, eL, eR, nf, x0, y0, un, ax, kd, dt);
}

// Persistent variant: each CTA takes tiles from a queue (an atomic counter per
// launch; two counters alternate, and each launch zeroes the next one's) into
// NBUF staging buffers.  Thread 0 loads a tile's u and psi boxes by two 2-D
// tensor copies (one box of DLX x DLY each, starting at (x0 - 8, y0 - 2)) that
// complete on the buffer's mbarrier; the buffer's next tile is claimed and its
// copy issued as soon as the buffer is free, so with NBUF = 2 it lands while
// this CTA computes the other buffer's tile.
// Boxes reaching past the grid's edge are zero-filled by the copy; the threads
// then put in the periodic images from global memory.  A wait that runs out
// (about a second) latches MLSD_ETIMEOUT into g_dns_status and ends the CTA's
// walk after a second bounded wait for each copy it has issued.
__device__ int g_dns_status;

template <int DTY, int NBUF>
struct DnsTma {
    static constexpr int DLY = DnsTile<DTY>::DLY;
    static constexpr int FIELD = DLY * DLX;                        // floats per staged field
    static constexpr int BUF = (2 * FIELD * 4 + 1023) / 1024 * 256; // floats per buffer (1 KB steps)
    static constexpr size_t SMEM = 1024 + (size_t)NBUF * BUF * 4 + (size_t)2 * DTY * DG * 4;
    static constexpr uint32_t BYTES = 2u * FIELD * 4u;              // one tile's copies
};

template <int DTY, int NBUF, bool PAIR>
__global__ void __launch_bounds__(DnsTile<DTY>::DTH)
k_dns_tma(const __grid_constant__ CUtensorMap mu, const __grid_constant__ CUtensorMap mp, int nf,
          const float *__restrict__ u, const float *__restrict__ psi, float *__restrict__ un,
          float ax, float kd, float dt, int *queue, int which)
{
    using T = DnsTma<DTY, NBUF>;
    constexpr int DLY = T::DLY, DTH = DnsTile<DTY>::DTH;
    extern __shared__ __align__(16) unsigned char dsm_raw[];
    __shared__ __align__(8) uint64_t full[NBUF];
    __shared__ int tile_of[NBUF];
    // the copies land at 1 KB-aligned buffers
    float *base = reinterpret_cast<float *>(dsm_raw + ((1024 - (smem_addr(dsm_raw) & 1023)) & 1023));
    float *eL = base + NBUF * T::BUF, *eR = eL + DTY * DG;
    const int tiles_x = nf / DTX, ntiles = tiles_x * (nf / DTY);
    const CUtensorMap *pmu = &mu, *pmp = &mp;
    // claim the next tile of the launch for buffer b and start its copies; past the
    // last tile, a plain arrival completes the phase so that the CTA's wait ends
    auto claim = [&](int b) {
        const int t = atomicAdd(&queue[which], 1);
        tile_of[b] = t;
        const uint32_t mb = smem_addr(&full[b]);
        if (t < ntiles) {
            const int x0 = (t % tiles_x) * DTX, y0 = (t / tiles_x) * DTY;
            float *su = base + b * T::BUF;
            mbar_expect(mb, T::BYTES);
            tma_load_2d(smem_addr(su), pmu, x0 - 8, y0 - 2, mb);
            tma_load_2d(smem_addr(su + T::FIELD), pmp, x0 - 8, y0 - 2, mb);
        } else {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(mb) : "memory");
        }
    };
    if (threadIdx.x == 0) {
        for (int b = 0; b < NBUF; ++b) mbar_init1(smem_addr(&full[b]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (blockIdx.x == 0) queue[which ^ 1] = 0;      // the next launch's queue
        for (int b = 0; b < NBUF; ++b) claim(b);
    }
    __syncthreads();                                     // the mbarriers are initialised
    for (int k = 0;; ++k) {
        const int b = k % NBUF;
        const uint32_t mb = smem_addr(&full[b]), par = (uint32_t)((k / NBUF) & 1);
        const bool ok = mbar_wait_bounded(mb, par);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicCAS(&g_dns_status, 0, MLSD_ETIMEOUT);
                // the copies of this and the other buffers, if still coming
                for (int j = 0; j < NBUF; ++j)
                    if (tile_of[(k + j) % NBUF] < ntiles)
                        mbar_wait_bounded(smem_addr(&full[(k + j) % NBUF]),
                                          (uint32_t)(((k + j) / NBUF) & 1));
            }
            break;
        }
        const int t = tile_of[b];
        if (t >= ntiles) break;                         // claims only grow: no copy is pending
        const int x0 = (t % tiles_x) * DTX, y0 = (t / tiles_x) * DTY;
        float *su = base + b * T::BUF, *sp = su + T::FIELD;
        if (x0 == 0 || x0 + DTX == nf || y0 == 0 || y0 + DTY == nf) {
            // periodic images of the staged cells outside the grid
            for (int e = threadIdx.x; e < DLY * DLX; e += DTH) {
                const int r = e / DLX, c = e % DLX;
                int gy = y0 - 2 + r, gx = x0 - 8 + c;
                if (gy >= 0 && gy < nf && gx >= 0 && gx < nf) continue;
                gy = gy < 0 ? gy + nf : (gy >= nf ? gy - nf : gy);
                gx = gx < 0 ? gx + nf : (gx >= nf ? gx - nf : gx);
                su[e] = u[(long long)gy * nf + gx];
                sp[e] = psi[(long long)gy * nf + gx];
            }
            __syncthreads();
        }
        if constexpr (PAIR) dns_tile2<DTY>(su, sp, eL, eR, nf, x0, y0, un, ax, kd, dt);
        else dns_tile<DTY>(su, sp, eL, eR, nf, x0, y0, un, ax, kd, dt);
        // every thread's reads and writes of this buffer come before the next copy into it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) claim(b);
    }
}

// Failure-path check of the tile wait: one thread waits on a fresh mbarrier that
// receives no arrival and no copy, so the wait runs out and latches MLSD_ETIMEOUT
__global__ void k_wait_check_tile(int *status)
{
    __shared__ __align__(8) uint64_t mb;
    if (threadIdx.x == 0) {
        mbar_init1(smem_addr(&mb));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!mbar_wait_bounded(smem_addr(&mb), 0)) atomicCAS(status, 0, MLSD_ETIMEOUT);
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

// the two tile counters of the persistent kernels, per device (zeroed once), and
// which one the next launch on that device takes (every persistent launch, of any
// tile shape, alternates them: each launch zeroes the other for its successor)
static std::vector<int> g_dns_which;
// the two tile counters of the persistent kernels, per device (zeroed once)
static cudaError_t dns_queue(int dev, cudaStream_t s, int **out, int *which)
{
    static std::mutex mu;
    static std::vector<int *> q;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)q.size() <= dev) q.resize(dev + 1, nullptr);
    if ((int)g_dns_which.size() <= dev) g_dns_which.resize(dev + 1, 0);
    if (!q[dev]) {
        cudaError_t e = cudaMalloc((void **)&q[dev], 2 * sizeof(int));
        if (e == cudaSuccess) e = cudaMemsetAsync(q[dev], 0, 2 * sizeof(int), s);
        if (e != cudaSuccess) { q[dev] = nullptr; return e; }
    }
    *out = q[dev];
    *which = g_dns_which[dev];
    g_dns_which[dev] ^= 1;
    return cudaSuccess;
}

template <int DTY, int NBUF, bool PAIR = false>
static cudaError_t dns_launch_tma(int nf, const CUtensorMap &ma, const CUtensorMap &mp,
                                  const float *a, const float *psi, float *b, float ax, float kd,
                                  float dt, cudaStream_t s)
{
    using T = DnsTma<DTY, NBUF>;
    constexpr int DTH = DnsTile<DTY>::DTH;
    const void *fn = reinterpret_cast<const void *>(&k_dns_tma<DTY, NBUF, PAIR>);
    static std::mutex mu;
    static std::vector<int> per_sm;                 // resident CTAs per SM, by device
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int res = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if ((int)per_sm.size() <= dev) per_sm.resize(dev + 1, 0);
        if (per_sm[dev] == 0) {
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::SMEM);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[dev], fn, DTH, T::SMEM);
            if (e != cudaSuccess) return e;
            if (per_sm[dev] < 1) return cudaErrorInvalidConfiguration;
        }
        res = per_sm[dev];
    }
    const long long ntiles = (long long)(nf / DTX) * (nf / DTY);
    const int grid = (int)std::min<long long>(ntiles, (long long)res * sms);
    int *queue = nullptr, which = 0;                 // launches alternate the two counters
    e = dns_queue(dev, s, &queue, &which);
    if (e != cudaSuccess) return e;
    k_dns_tma<DTY, NBUF, PAIR><<<grid, DTH, T::SMEM, s>>>(ma, mp, nf, a, psi, b, ax, kd, dt, queue,
                                                          which);
    return cudaGetLastError();
}

// DNS kernel variants: per-tile CTAs staged by cp.async (tile height 64 rows, 2 CTAs/SM,
// or 32 rows, 4 CTAs/SM), or persistent CTAs fed by tensor copies (32 rows with one or
// two staging buffers, 64 rows with one; 32 rows with the f32x2 pair arithmetic).
// Picked once per process by timing each on the caller's grid;
// MLSD_DNS_TY = 64 | 32 | t32 | t32x2 | t64 | t32p pins one.
enum DnsKind { kCp64, kCp32, kTma32, kTma32x2, kTma64, kTma32p, kDnsKinds };
static int g_dns_kind = -1;

static cudaError_t dns_launch_kind(int kind, int nf, const CUtensorMap *maps, int ia,
                                   const float *a, const float *psi, float *b, float ax, float kd,
                                   float dt, cudaStream_t s)
{
    switch (kind) {
    case kCp64: return dns_launch<64>(nf, a, psi, b, ax, kd, dt, s);
    case kCp32: return dns_launch<32>(nf, a, psi, b, ax, kd, dt, s);
    case kTma32: return dns_launch_tma<32, 1>(nf, maps[ia], maps[2], a, psi, b, ax, kd, dt, s);
    case kTma32x2: return dns_launch_tma<32, 2>(nf, maps[ia], maps[2], a, psi, b, ax, kd, dt, s);
    case kTma64: return dns_launch_tma<64, 1>(nf, maps[ia], maps[2], a, psi, b, ax, kd, dt, s);
    case kTma32p:
        return dns_launch_tma<32, 1, true>(nf, maps[ia], maps[2], a, psi, b, ax, kd, dt, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t dns_run(int nf, float *u, float *u_tmp, const float *psi, double kappa, double dt,
                    int nsteps, cudaStream_t s)
{
    const double h = 2.0 * kPi / nf;
    const float ax = (float)(1.0 / (2.0 * h));
    const float kd = (float)(kappa / (h * h));
    // tensor maps of u, u_tmp and psi; boxes of DLX x (DTY + 4), one map set per tile height
    CUtensorMap m32[3], m64[3];
    const bool tma = encode_f32_2d(&m32[0], u, nf, nf, DLX, 36) &&
                     encode_f32_2d(&m32[1], u_tmp, nf, nf, DLX, 36) &&
                     encode_f32_2d(&m32[2], psi, nf, nf, DLX, 36) &&
                     encode_f32_2d(&m64[0], u, nf, nf, DLX, 68) &&
                     encode_f32_2d(&m64[1], u_tmp, nf, nf, DLX, 68) &&
                     encode_f32_2d(&m64[2], psi, nf, nf, DLX, 68);
    auto maps_of = [&](int kind) -> const CUtensorMap * { return kind == kTma64 ? m64 : m32; };
    if (const char *env = std::getenv("MLSD_DNS_TY")) {
        const std::string v(env);
        g_dns_kind = v == "32" ? kCp32 : v == "t32" ? kTma32 : v == "t32x2" ? kTma32x2
                   : v == "t64" ? kTma64 : v == "t32p" ? kTma32p : kCp64;
    }
    if (!tma && g_dns_kind >= kTma32) g_dns_kind = kCp32;
    if (g_dns_kind < 0 && nsteps > 0) {
        // one trial step of each into u_tmp (u is not modified), best of two
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        for (int kind = 0; kind < (tma ? (int)kDnsKinds : (int)kTma32); ++kind) {
            float t = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, s);
                cudaError_t e = dns_launch_kind(kind, nf, maps_of(kind), 0, u, psi, u_tmp, ax, kd,
                                                (float)dt, s);
                cudaEventRecord(e1, s);
                if (e != cudaSuccess) return e;
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) t = std::min(t, ms);
            }
            count_launches(3);
            if (t < best) { best = t; g_dns_kind = kind; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    float *a = u, *b = u_tmp;
    int ia = 0;
    count_launches(nsteps);
    for (int st = 0; st < nsteps; ++st) {
        cudaError_t e = dns_launch_kind(g_dns_kind, nf, maps_of(g_dns_kind), ia, a, psi, b, ax, kd,
                                        (float)dt, s);
        if (e != cudaSuccess) return e;
        float *t = a; a = b; b = t;
        ia ^= 1;
    }
    if (a != u)
        return cudaMemcpyAsync(u, a, (size_t)nf * nf * sizeof(float), cudaMemcpyDeviceToDevice, s);
    return cudaGetLastError();
}

const char *dns_kernel_name()
{
    static const char *names[kDnsKinds] = {"k_dns_step<64>", "k_dns_step<32>", "k_dns_tma<32,1>",
                                           "k_dns_tma<32,2>", "k_dns_tma<64,1>",
                                           "k_dns_tma<32,1,pairs>"};
    return g_dns_kind < 0 ? "" : names[g_dns_kind];
}

int dns_status_take(cudaStream_t s)
{
    int v = 0;
    const int zero = 0;
    if (cudaMemcpyFromSymbolAsync(&v, g_dns_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyToSymbolAsync(g_dns_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return MLSD_ECUDA;
    return v;
}

cudaError_t launch_wait_check_tile(int *status, cudaStream_t s)
{
    count_launches(1);
    k_wait_check_tile<<<1, 32, 0, s>>>(status);
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
