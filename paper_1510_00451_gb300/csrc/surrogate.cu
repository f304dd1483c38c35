// Learned surrogate of the patch solve (not part of the paper's method; the
// plain patch solve stays its fallback and the reference for its error).
//
// Features: per patch, the 17 x 17 low-mode DFT of the patch's band psi (patch
// mean removed) times MLSD_SUR_PSI_SCALE / (tr(B)/2), then B/kappa, log kappa
// (k_features), and the perturbation moments T_2..T_6 of the steady corrector
// equation with the [2/2], [3/3], [4/4] Pade approximants of its resummed
// series (from T_2..T_19), each as asinh(MLSD_SUR_T_SCALE x / tr B) (k_series):
// 606 values stored as one bfloat16 row of MLSD_SUR_IN (640, zero padded).
// Network: an ensemble of members, each 640 -> h -> h -> h -> 3 with the exact
// erf GELU, bfloat16 weights and activations, FP32 accumulation; output
// asinh((K - B - E) MLSD_SUR_Y_SCALE / tr(B)), E the [4/4] approximant.  Training
// kernels here run on the CUDA cores (FP32 FMA on bfloat16 operands); the
// inference forward has a tensor-core (tcgen05) kernel in mlp_tc.cu.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mlsd_internal.cuh"

namespace mlsd {
namespace {

constexpr int KMODE = 8;                   // local modes -8..8
constexpr int NMODE = 2 * KMODE + 1;       // 17

// ---------------------------------------------------------------------------
// Features 0..581 and the zero padding: one CTA per patch.  The features of an
// n x n patch are those of its nf x nf samples every sub-th node (nf = n / sub
// <= 64: the samples are staged in shared memory)
__global__ void k_features(const float *band, long long Nl, long long tile, int n, int sub,
                           int n_macro, const int *pidx, long long count, const double *B,
                           double kappa, __nv_bfloat16 *X, float *F32)
{
    const int nf = n / sub;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *psi = reinterpret_cast<float *>(smem_raw);              // [nf][nf]
    float2 *Fr = reinterpret_cast<float2 *>(psi + nf * nf);        // [nf][17] row transforms
    __shared__ double red[32];
    __shared__ float2 tw[64];                                      // e^{-2 pi i r / nf}
    const long long item = blockIdx.x;
    if (item >= count) return;
    const long long p = pidx ? (long long)pidx[item] : item;
    const long long ox = patch_origin(p % n_macro, n_macro, Nl, n);
    const long long oy = patch_origin(p / n_macro, n_macro, Nl, n);
    double sum = 0.0;
    for (int c = threadIdx.x; c < nf * nf; c += blockDim.x) {
        const int b = c / nf, a = c % nf;
        const float v = patch_band(band, Nl, tile, p, ox, oy, n, a * sub, b * sub);
        psi[c] = v;
        sum += v;
    }
    for (int r = threadIdx.x; r < nf; r += blockDim.x) {
        float s, c;
        sincospif(-2.0f * (float)r / (float)nf, &s, &c);
        tw[r] = make_float2(c, s);
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    const float mean = (float)(tot / ((double)nf * nf));
    // rows: Fr[b][k1] = sum_a (psi - mean) e^{-2 pi i k1 a / nf}
    for (int t = threadIdx.x; t < nf * NMODE; t += blockDim.x) {
        const int b = t / NMODE, k1 = t % NMODE - KMODE;
        float sr = 0.f, si = 0.f;
        const int step = (int)pmod_ll((long long)k1, nf);
        int r = 0;
        for (int a = 0; a < nf; ++a) {
            const float2 w = tw[r];
            const float v = psi[b * nf + a] - mean;
            sr = fmaf(v, w.x, sr);
            si = fmaf(v, w.y, si);
            r += step;
            if (r >= nf) r -= nf;
        }
        Fr[t] = make_float2(sr, si);
    }
    __syncthreads();
    const double B11 = B[3 * p], B12 = B[3 * p + 1], B22 = B[3 * p + 2];
    const double trh = 0.5 * (B11 + B22);
    const float scale = (float)(MLSD_SUR_PSI_SCALE / ((double)nf * nf * trh));
    __nv_bfloat16 *xr = X + item * (long long)MLSD_SUR_IN;
    float *fr = F32 ? F32 + item * (long long)MLSD_SUR_FEATURES : nullptr;
    for (int t = threadIdx.x; t < NMODE * NMODE; t += blockDim.x) {
        const int k2 = t / NMODE - KMODE, k1i = t % NMODE;
        float sr = 0.f, si = 0.f;
        const int step = (int)pmod_ll((long long)k2, nf);
        int r = 0;
        for (int b = 0; b < nf; ++b) {
            const float c = tw[r].x, s = tw[r].y;
            r += step;
            if (r >= nf) r -= nf;
            const float2 f = Fr[b * NMODE + k1i];
            // (f.x + i f.y)(c + i s)
            sr += f.x * c - f.y * s;
            si += f.x * s + f.y * c;
        }
        const float re = sr * scale, im = si * scale;
        xr[2 * t] = __float2bfloat16_rn(re);
        xr[2 * t + 1] = __float2bfloat16_rn(im);
        if (fr) { fr[2 * t] = re; fr[2 * t + 1] = im; }
    }
    const int t = 2 * NMODE * NMODE + threadIdx.x;
    if (t < MLSD_SUR_IN && (t < 582 || t >= MLSD_SUR_FEATURES)) {   // 582..605: k_series
        float v = 0.f;
        if (t == 578) v = (float)(B11 / kappa);
        else if (t == 579) v = (float)(B12 / kappa);
        else if (t == 580) v = (float)(B22 / kappa);
        else if (t == 581) v = (float)log(kappa);
        xr[t] = __float2bfloat16_rn(v);
        if (fr && t < MLSD_SUR_FEATURES) fr[t] = v;
    }
}

// ---------------------------------------------------------------------------
// Perturbation moments of the steady corrector equation (features 582..605 and
// the baseline E of the network's target).  In index units (h = 1; the moments
// do not depend on h):
//   v1 = -(psi[b+1][a] - psi[b-1][a]) / 2,  v2 = (psi[b][a+1] - psi[b][a-1]) / 2,
//   g(k) = 1 / D(k), D = B11 (2 - 2 cos t1) + B22 (2 - 2 cos t2) + 2 B12 sin t1 sin t2,
//   g(0) = 0 (-L0^{-1} is multiplication of the DFT by g),
//   c_j^0 = -L0^{-1} v_j,  c_j^m = -L0^{-1} (v1 D0x + v2 D0y) c_j^{m-1},
//   T_m = sym <v_i c_j^{m-2}>  (m = 2..19; means over the cells summed in FP32
//   per thread and per warp, in FP64 across the warps).
// Both fields go through one complex FFT as c1 + i c2: g is real and even in
// k, so multiplying the transform of (f1 + i f2) by g transforms each part.
// One CTA of 256 threads per patch, everything in shared memory: the complex
// work field, v1, v2, c1, c2, the symbol g and the twiddles (n = 32: 28 KB,
// n = 64: 112 KB).  Radix-2 FFT along rows, then columns, in FP32.
// Resummation (FP64, one thread per component): pairs p_k = T_(2k+2) + T_(2k+3),
// k = 0..8, and the [K/K] Pade approximants at 1 of sum_k p_k x^k by Wynn's
// epsilon algorithm on the partial sums (K = 2, 3, 4); E = [4/4] and
// Eout[item] = (E11, E12, E22, max_c |[4/4]_c - [3/3]_c|).
template <int N>
__device__ void fft2_smem(float2 *z, const float2 *tw, bool inverse)
{
    constexpr int LOG = N == 32 ? 5 : 6;
    for (int pass = 0; pass < 2; ++pass) {
        // rows: consecutive threads take consecutive elements of a row; columns:
        // consecutive threads take consecutive columns (no shared-memory bank conflicts
        // on the strided column accesses)
        const int es = pass == 0 ? 1 : N, ls = pass == 0 ? N : 1;
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
            const int line = pass == 0 ? e / N : e % N, i = pass == 0 ? e % N : e / N;
            const int r = (int)(__brev((unsigned)i) >> (32 - LOG));
            if (i < r) {
                const float2 a = z[line * ls + i * es];
                z[line * ls + i * es] = z[line * ls + r * es];
                z[line * ls + r * es] = a;
            }
        }
        __syncthreads();
        for (int half = 1; half < N; half <<= 1) {
            const int tws = N / (2 * half);
            for (int t = threadIdx.x; t < N * N / 2; t += blockDim.x) {
                const int line = pass == 0 ? t / (N / 2) : t % N;
                const int j = pass == 0 ? t % (N / 2) : t / N;
                const int pos = j & (half - 1), grp = j / half;
                const int i0 = grp * 2 * half + pos, i1 = i0 + half;
                float2 w = tw[pos * tws];
                if (inverse) w.y = -w.y;
                const float2 a = z[line * ls + i0 * es], b = z[line * ls + i1 * es];
                const float2 bw = make_float2(b.x * w.x - b.y * w.y, b.x * w.y + b.y * w.x);
                z[line * ls + i0 * es] = make_float2(a.x + bw.x, a.y + bw.y);
                z[line * ls + i1 * es] = make_float2(a.x - bw.x, a.y - bw.y);
            }
            __syncthreads();
        }
    }
}

// block sum of 4 doubles (256 threads = 8 warps); every thread gets the totals
__device__ __forceinline__ void block_sum4(double (&v)[4], double (*red)[8])
{
#pragma unroll
    for (int q = 0; q < 4; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 4; ++q) red[q][threadIdx.x >> 5] = v[q];
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[q][w];
        v[q] = t;
    }
    __syncthreads();
}

// block sum of 4 floats into 4 doubles held by thread 0 only: FP32 within a
// thread and across the warp, FP64 for the 8 warp partials (the FP64 pipe of
// this part is narrow, so the per-thread and per-warp sums stay in FP32)
__device__ __forceinline__ void block_sum4_root(float (&v)[4], double (*red)[8], double (&out)[4])
{
#pragma unroll
    for (int q = 0; q < 4; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 4; ++q) red[q][threadIdx.x >> 5] = (double)v[q];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) {
            double t = 0.0;
            for (int w = 0; w < 8; ++w) t += red[q][w];
            out[q] = t;
        }
}

// [K/K] at 1 of sum_k c_k x^k by Wynn's epsilon algorithm on the partial sums
// (c_0..c_2K, K <= 4); where a difference vanishes, the last even column reached
__device__ double wynn_dev(const double *c, int K)
{
    double ea[10], eb[10];
    double *prev = ea, *cur = eb;
    const int n = 2 * K + 1;
    double acc = 0.0;
    for (int j = 0; j < n; ++j) { acc += c[j]; cur[j] = acc; prev[j] = 0.0; }
    prev[n] = 0.0;
    double best = cur[n - 1];
    int len = n;
    for (int k = 1; k <= 2 * K; ++k) {
        for (int j = 0; j < len - 1; ++j) {          // in place: prev[j] <- eps_{k}^{(j)}
            const double d = cur[j + 1] - cur[j];
            if (fabs(d) < 1e-300) return best;
            prev[j] = prev[j + 1] + 1.0 / d;
        }
        double *t = prev; prev = cur; cur = t;
        len -= 1;
        if ((k & 1) == 0) best = cur[0];
    }
    return cur[0];
}

constexpr int SERIES_M = 19;               // moments T_2..T_19

template <int N>
__global__ void __launch_bounds__(256) k_series(const float *band, long long Nl, long long tile,
                                                int n, int sub, int n_macro, const int *pidx,
                                                long long count, const double *B,
                                                __nv_bfloat16 *X, float *F32, double *Eout)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *z = reinterpret_cast<float2 *>(smem_raw);               // [N][N] complex
    float *v1 = reinterpret_cast<float *>(z + N * N);                // [N][N] each:
    float *v2 = v1 + N * N, *c1 = v2 + N * N, *c2 = c1 + N * N;      // velocity, iterates,
    float *g = c2 + N * N;                                           // 1 / D(k)
    float2 *tw = reinterpret_cast<float2 *>(g + N * N);              // [N/2]
    float *psi = c1;                                                 // psi until v is formed
    __shared__ double red[4][8];
    __shared__ double Tm[SERIES_M - 1][3];
    const long long item = blockIdx.x;
    if (item >= count) return;
    const long long p = pidx ? (long long)pidx[item] : item;
    const long long ox = patch_origin(p % n_macro, n_macro, Nl, n);
    const long long oy = patch_origin(p / n_macro, n_macro, Nl, n);
    const double B11 = B[3 * p], B12 = B[3 * p + 1], B22 = B[3 * p + 2];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int b = e / N, a = e % N;
        const float v = patch_band(band, Nl, tile, p, ox, oy, n, a * sub, b * sub);
        psi[e] = v;
        acc[0] += v;
        // the symbol of -L0^{-1}, once per patch
        float s1, co1, s2, co2;
        sincospif(2.0f * (float)a / (float)N, &s1, &co1);
        sincospif(2.0f * (float)b / (float)N, &s2, &co2);
        const float D = (float)B11 * (2.f - 2.f * co1) + (float)B22 * (2.f - 2.f * co2)
                        + 2.f * (float)B12 * s1 * s2;
        g[e] = e == 0 ? 0.f : 1.f / D;
    }
    for (int k = threadIdx.x; k < N / 2; k += blockDim.x) {
        float sn, cs;
        sincospif(-2.0f * (float)k / (float)N, &sn, &cs);
        tw[k] = make_float2(cs, sn);
    }
    block_sum4(acc, red);
    const float mean = (float)(acc[0] / (double)(N * N));
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int b = e / N, a = e % N;
        const int ap = (a + 1) & (N - 1), am = (a + N - 1) & (N - 1);
        const int bp = (b + 1) & (N - 1), bm = (b + N - 1) & (N - 1);
        v1[e] = 0.5f * (psi[bm * N + a] - psi[bp * N + a]);
        v2[e] = 0.5f * (psi[b * N + ap] - psi[b * N + am]);
        z[e] = make_float2(psi[e] - mean, 0.f);
    }
    __syncthreads();
    fft2_smem<N>(z, tw, false);
    // c^0: transform of c1 + i c2 = g (-s1 - i s2) psihat
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int k1 = e % N, k2 = e / N;
        const float s1 = sinpif(2.0f * (float)k1 / (float)N), s2 = sinpif(2.0f * (float)k2 / (float)N);
        const float2 q = z[e];
        z[e] = make_float2(g[e] * (-q.x * s1 + q.y * s2), g[e] * (-q.x * s2 - q.y * s1));
    }
    __syncthreads();
    fft2_smem<N>(z, tw, true);
    const float inv = 1.0f / (float)(N * N);
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) { c1[e] = z[e].x * inv; c2[e] = z[e].y * inv; }
    __syncthreads();
    for (int m = 2; m <= SERIES_M; ++m) {
        float sm[4] = {0.f, 0.f, 0.f, 0.f};
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
            const float a1 = v1[e], a2 = v2[e];
            sm[0] = fmaf(a1, c1[e], sm[0]); sm[1] = fmaf(a1, c2[e], sm[1]);
            sm[2] = fmaf(a2, c1[e], sm[2]); sm[3] = fmaf(a2, c2[e], sm[3]);
            if (m < SERIES_M) {
                const int b = e / N, a = e % N;
                const int ap = (a + 1) & (N - 1), am = (a + N - 1) & (N - 1);
                const int bp = (b + 1) & (N - 1), bm = (b + N - 1) & (N - 1);
                const float d1x = 0.5f * (c1[b * N + ap] - c1[b * N + am]);
                const float d1y = 0.5f * (c1[bp * N + a] - c1[bm * N + a]);
                const float d2x = 0.5f * (c2[b * N + ap] - c2[b * N + am]);
                const float d2y = 0.5f * (c2[bp * N + a] - c2[bm * N + a]);
                z[e] = make_float2(fmaf(a1, d1x, a2 * d1y), fmaf(a1, d2x, a2 * d2y));
            }
        }
        double tot[4];
        block_sum4_root(sm, red, tot);
        if (threadIdx.x == 0) {
            const double nn = (double)(N * N);
            Tm[m - 2][0] = tot[0] / nn;
            Tm[m - 2][1] = 0.5 * (tot[1] + tot[2]) / nn;
            Tm[m - 2][2] = tot[3] / nn;
        }
        if (m == SERIES_M) break;
        fft2_smem<N>(z, tw, false);
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
            const float q = g[e];
            z[e] = make_float2(z[e].x * q, z[e].y * q);
        }
        __syncthreads();
        fft2_smem<N>(z, tw, true);
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) { c1[e] = z[e].x * inv; c2[e] = z[e].y * inv; }
        __syncthreads();
    }
    __syncthreads();
    const double sc = MLSD_SUR_T_SCALE / (B11 + B22);
    __nv_bfloat16 *xr = X + item * (long long)MLSD_SUR_IN;
    float *fr = F32 ? F32 + item * (long long)MLSD_SUR_FEATURES : nullptr;
    if (threadIdx.x < 3) {
        const int c = threadIdx.x;
        double pk[9];
        for (int k = 0; k < 9; ++k) pk[k] = Tm[2 * k][c] + Tm[2 * k + 1][c];
        const double P2 = wynn_dev(pk, 2), P3 = wynn_dev(pk, 3), E = wynn_dev(pk, 4);
        red[0][c] = fabs(E - P3);
        if (Eout) Eout[item * 4 + c] = E;
        const float f2 = (float)asinh(sc * P2), f3 = (float)asinh(sc * P3),
                    fe = (float)asinh(sc * E);
        xr[597 + c] = __float2bfloat16_rn(f2);
        xr[600 + c] = __float2bfloat16_rn(f3);
        xr[603 + c] = __float2bfloat16_rn(fe);
        if (fr) { fr[597 + c] = f2; fr[600 + c] = f3; fr[603 + c] = fe; }
    }
    if (threadIdx.x < 15) {
        const float f = (float)asinh(sc * Tm[threadIdx.x / 3][threadIdx.x % 3]);
        xr[582 + threadIdx.x] = __float2bfloat16_rn(f);
        if (fr) fr[582 + threadIdx.x] = f;
    }
    __syncthreads();
    if (threadIdx.x == 0 && Eout) {
        const double g0 = fmax(red[0][0], fmax(red[0][1], red[0][2]));
        Eout[item * 4 + 3] = (red[0][0] == red[0][0] && red[0][1] == red[0][1] &&
                              red[0][2] == red[0][2]) ? g0 : red[0][0] + red[0][1] + red[0][2];
    }
}

// ---------------------------------------------------------------------------
// Periodic component of a patch's band samples u (periodic-plus-smooth
// decomposition, Moisan 2011): the boundary image v is nonzero on the border
// samples only, v(x) = sum over the seam neighbours y of u(y) - u(x); s solves
// the periodic 5-point Poisson problem Lap s = v (symbol 2 cos t1 + 2 cos t2 - 4,
// zero mean); p = u - s goes to the patch's tile.  One CTA of 256 threads per
// patch, FFTs in shared memory (FP32).
template <int N>
__global__ void __launch_bounds__(256) k_periodize(const float *band, long long Nl, int n_macro,
                                                   const int *pidx, long long count, float *tiles)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *z = reinterpret_cast<float2 *>(smem_raw);               // [N][N] complex
    float *u = reinterpret_cast<float *>(z + N * N);                 // [N][N]
    float2 *tw = reinterpret_cast<float2 *>(u + N * N);              // [N/2]
    const long long item = blockIdx.x;
    if (item >= count) return;
    const long long p = pidx ? (long long)pidx[item] : item;
    const long long ox = patch_origin(p % n_macro, n_macro, Nl, N);
    const long long oy = patch_origin(p / n_macro, n_macro, Nl, N);
    for (int e = threadIdx.x; e < N * N; e += blockDim.x)
        u[e] = band[pmod_ll(oy + e / N, Nl) * Nl + pmod_ll(ox + e % N, Nl)];
    for (int k = threadIdx.x; k < N / 2; k += blockDim.x) {
        float sn, cs;
        sincospif(-2.0f * (float)k / (float)N, &sn, &cs);
        tw[k] = make_float2(cs, sn);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int b = e / N, a = e % N;
        float v = 0.f;
        if (b == 0) v += u[(N - 1) * N + a] - u[a];
        if (b == N - 1) v += u[a] - u[(N - 1) * N + a];
        if (a == 0) v += u[b * N + N - 1] - u[b * N];
        if (a == N - 1) v += u[b * N] - u[b * N + N - 1];
        z[e] = make_float2(v, 0.f);
    }
    __syncthreads();
    fft2_smem<N>(z, tw, false);
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        float s1, c1, s2, c2;
        sincospif(2.0f * (float)(e % N) / (float)N, &s1, &c1);
        sincospif(2.0f * (float)(e / N) / (float)N, &s2, &c2);
        const float d = 2.f * c1 + 2.f * c2 - 4.f;
        z[e] = e == 0 ? make_float2(0.f, 0.f) : make_float2(z[e].x / d, z[e].y / d);
    }
    __syncthreads();
    fft2_smem<N>(z, tw, true);
    const float inv = 1.0f / (float)(N * N);
    float *t = tiles + p * (long long)(N * N);
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) t[e] = u[e] - z[e].x * inv;
}

// ---------------------------------------------------------------------------
// CUDA-core GEMM with bfloat16 or FP32 operands and FP32 accumulation:
//   C[i][j] = sum_k A(i, k) B(k, j) (+ bias[j]) (+ C[i][j] if accumulate)
// A(i, k) = A[i * sam + k * sak], B(k, j) = B[k * sbk + j * sbn].
// Optional epilogue: act[i][j] = bf16(gelu(C[i][j])).
__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }

__device__ __forceinline__ float gelu_f(float z)
{
    return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_d(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

constexpr int GK = 16;          // k depth of one shared-memory stage
constexpr int SPLIT_MAX = 16;   // most k splits of one GEMM

// Epilogue of the GEMM and of its split-k reduction, applied to output (i, j) in order:
// + bias[j]; + the old C(i, j) (accumulate); times gelu'(dgelu(i, j)) (the backward GELU,
// dgelu shares C's row stride), rounded to a bfloat16 value (the hidden layers' dZ are
// bfloat16 operands of the backward contractions); store C; act(i, j) = gelu(C(i, j)) in
// bfloat16.
struct Epi {
    const float *bias = nullptr;
    int accumulate = 0;
    const float *dgelu = nullptr;
    __nv_bfloat16 *act = nullptr;
    long long sactm = 0;
};

__device__ __forceinline__ void epilogue(const Epi &e, float v, int gi, int gj, float *C,
                                         long long scm)
{
    if (e.bias) v += e.bias[gj];
    if (e.accumulate) v += C[gi * scm + gj];
    if (e.dgelu) v = __bfloat162float(__float2bfloat16_rn(v * gelu_d(e.dgelu[gi * scm + gj])));
    C[gi * scm + gj] = v;
    if (e.act) e.act[gi * e.sactm + gj] = __float2bfloat16_rn(gelu_f(v));
}

// C[M x N] = A[M x K] B[K x N] on the CUDA cores with FP32 accumulation, where
// A(i, k) = A[i sam + k sak] and B(k, j) = B[k sbk + j sbn]. Either operand may have either
// index contiguous; the tile loads run along the contiguous one, so every warp's global
// reads are coalesced. One T x T output tile per CTA of 256 threads: thread (tx, ty) owns
// rows 4 ty + 64 a + (0..3) and columns 4 tx + 64 b + (0..3), read from shared memory as
// float4. The next k stage is loaded into registers while the current one is multiplied.
// With gridDim.z > 1 the CTA sums only k in [z kc, (z + 1) kc) and stores its raw partial
// at C + z scz (row stride scm); k_split_reduce adds the partials and applies the epilogue.
// With RS, the CTAs of the first column tile also sum A's rows over their k range into
// rs[z M + i] (the bias gradient, when A is the transposed output gradient). That variant
// is capped to keep 3 CTAs per SM; the plain one reaches it uncapped.
template <typename TA, typename TB, int T, bool RS = false>
__global__ void __launch_bounds__(256, RS ? 3 : 0)
    k_gemm(int M, int N, int K, int kc, const TA *A, long long sam, long long sak, const TB *Bm,
           long long sbk, long long sbn, float *C, long long scm, long long scz, Epi ep, float *rs)
{
    constexpr int R = T / 16, E = T * GK / 256;
    __shared__ __align__(16) float As[GK][T + 4];
    __shared__ __align__(16) float Bs[GK][T + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int i0 = blockIdx.y * T, j0 = blockIdx.x * T;
    const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
    const bool a_rows = sam == 1, b_cols = sbn == 1;
    float ra[E], rb[E];
    auto load = [&](int k0) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int t = threadIdx.x + 256 * e;
            const int r = a_rows ? t % T : t / GK, k = a_rows ? t / T : t % GK;
            const int gi = i0 + r, gk = k0 + k;
            ra[e] = (gi < M && gk < ke) ? to_f(A[gi * sam + gk * sak]) : 0.f;
            const int c = b_cols ? t % T : t / GK, q = b_cols ? t / T : t % GK;
            const int gj = j0 + c, gq = k0 + q;
            rb[e] = (gj < N && gq < ke) ? to_f(Bm[gq * sbk + gj * sbn]) : 0.f;
        }
    };
    float acc[R][R] = {};
    __shared__ float rsum[T];
    const bool rows_sum = RS && blockIdx.x == 0;
    if (rows_sum && threadIdx.x < T) rsum[threadIdx.x] = 0.f;
    if (kb < ke) load(kb);
    for (int k0 = kb; k0 < ke; k0 += GK) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int t = threadIdx.x + 256 * e;
            As[a_rows ? t / T : t % GK][a_rows ? t % T : t / GK] = ra[e];
            Bs[b_cols ? t / T : t % GK][b_cols ? t % T : t / GK] = rb[e];
        }
        __syncthreads();
        if (rows_sum && threadIdx.x < T) {
            float t = 0.f;
#pragma unroll
            for (int k = 0; k < GK; ++k) t += As[k][threadIdx.x];
            rsum[threadIdx.x] += t;
        }
        if (k0 + GK < ke) load(k0 + GK);
#pragma unroll
        for (int k = 0; k < GK; ++k) {
            float a[R], b[R];
#pragma unroll
            for (int q = 0; q < R / 4; ++q) {
                const float4 va = *reinterpret_cast<const float4 *>(&As[k][64 * q + 4 * ty]);
                const float4 vb = *reinterpret_cast<const float4 *>(&Bs[k][64 * q + 4 * tx]);
                a[4 * q] = va.x; a[4 * q + 1] = va.y; a[4 * q + 2] = va.z; a[4 * q + 3] = va.w;
                b[4 * q] = vb.x; b[4 * q + 1] = vb.y; b[4 * q + 2] = vb.z; b[4 * q + 3] = vb.w;
            }
#pragma unroll
            for (int q = 0; q < R; ++q)
#pragma unroll
                for (int r = 0; r < R; ++r) acc[q][r] = fmaf(a[q], b[r], acc[q][r]);
        }
        __syncthreads();
    }
    const bool split = gridDim.z > 1;
    if (rows_sum && threadIdx.x < T && i0 + (int)threadIdx.x < M)
        rs[blockIdx.z * M + i0 + threadIdx.x] = rsum[threadIdx.x];
    float *Cz = C + blockIdx.z * scz;
#pragma unroll
    for (int q = 0; q < R; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int gi = i0 + 64 * (q / 4) + 4 * ty + q % 4;
            const int gj = j0 + 64 * (r / 4) + 4 * tx + r % 4;
            if (gi >= M || gj >= N) continue;
            if (split) Cz[gi * scm + gj] = acc[q][r];
            else epilogue(ep, acc[q][r], gi, gj, C, scm);
        }
}

// C = sum over z = 0 .. S-1 of the partials ws[z M N + i N + j], in that order, then the
// epilogue; with rs, also rs[i] = sum over z of the row-sum partials rs_part[z M + i]
__global__ void k_split_reduce(int M, int N, int S, const float *ws, float *C, long long scm,
                               Epi ep, const float *rs_part, float *rs)
{
    const long long n = (long long)M * N, total = n + (rs ? M : 0);
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
         x += (long long)gridDim.x * blockDim.x) {
        float v = 0.f;
        if (x < n) {
            for (int z = 0; z < S; ++z) v += ws[z * n + x];
            epilogue(ep, v, (int)(x / N), (int)(x % N), C, scm);
        } else {
            for (int z = 0; z < S; ++z) v += rs_part[z * M + (x - n)];
            rs[x - n] = v;
        }
    }
}

int device_sms()
{
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            return 152;
        cache[dev] = n;
    }
    return cache[dev];
}

// CTAs of the 64-wide kernel resident on one SM (its registers decide), per device
template <typename TA, typename TB, bool RS>
int gemm_residency()
{
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!cache[dev]) {
        int r = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_gemm<TA, TB, 64, RS>, 256, 0) !=
                cudaSuccess || r < 1)
            r = 1;
        cache[dev] = r;
    }
    return cache[dev];
}

// One GEMM with its tiling: 128-wide tiles where they alone give every SM two CTAs, else
// 64-wide tiles, and where even those fill less than one wave of resident CTAs, k split over
// up to SPLIT_MAX CTAs (each at least 64 deep) whose partials go to ws (ws_n floats; no split
// without it).  With rs (length M), also rs[i] = sum over k of A(i, k).
template <typename TA, typename TB>
cudaError_t gemm(cudaStream_t s, int M, int N, int K, const TA *A, long long sam, long long sak,
                 const TB *B, long long sbk, long long sbn, float *C, long long scm, Epi ep,
                 float *ws, long long ws_n, float *rs = nullptr)
{
    const long long big = (long long)((M + 127) / 128) * ((N + 127) / 128);
    if (big >= 2LL * device_sms() && !rs) {
        count_launches(1);
        dim3 g((N + 127) / 128, (M + 127) / 128);
        k_gemm<TA, TB, 128><<<g, 256, 0, s>>>(M, N, K, K, A, sam, sak, B, sbk, sbn, C, scm, 0, ep,
                                              nullptr);
        return cudaGetLastError();
    }
    const long long slots = (long long)(rs ? gemm_residency<TA, TB, true>()
                                          : gemm_residency<TA, TB, false>()) * device_sms();
    const long long tiles = (long long)((M + 63) / 64) * ((N + 63) / 64);
    long long S = 1;
    if (ws && tiles < slots) {
        S = std::min<long long>({(long long)SPLIT_MAX, slots / tiles, K / 64});
        while (S > 1 && S * M * N + (rs ? S * M : 0) > ws_n) --S;
        S = std::max(S, 1LL);
    }
    const int kc = (int)((((K + S - 1) / S) + GK - 1) / GK * GK);
    S = std::max(1, (K + kc - 1) / kc);
    dim3 g((N + 63) / 64, (M + 63) / 64, (unsigned)S);
    count_launches(S > 1 ? 2 : 1);
    auto run64 = [&](int kc_, float *Cp, long long ldc, long long scz, Epi e, float *r) {
        if (r)
            k_gemm<TA, TB, 64, true><<<g, 256, 0, s>>>(M, N, K, kc_, A, sam, sak, B, sbk, sbn, Cp,
                                                       ldc, scz, e, r);
        else
            k_gemm<TA, TB, 64, false><<<g, 256, 0, s>>>(M, N, K, kc_, A, sam, sak, B, sbk, sbn, Cp,
                                                        ldc, scz, e, nullptr);
    };
    if (S == 1) {
        run64(K, C, scm, 0, ep, rs);
        return cudaGetLastError();
    }
    const long long n = (long long)M * N;
    float *rs_part = rs ? ws + S * n : nullptr;
    run64(kc, ws, N, n, Epi{}, rs_part);
    const long long nb = std::min<long long>((n + (rs ? M : 0) + 255) / 256, 8LL * device_sms());
    k_split_reduce<<<(unsigned)nb, 256, 0, s>>>(M, N, (int)S, ws, C, scm, ep, rs_part, rs);
    return cudaGetLastError();
}


// dZ4 = 2 (Z4 - Y) / (3 M), loss partial sums per block
__global__ void k_mse(int M, const float *Z4, const float *Y, float *dZ4, double *part)
{
    __shared__ double red[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < 3 * M) {
        const float d = Z4[i] - Y[i];
        dZ4[i] = 2.0f * d / (3.0f * (float)M);
        l = (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void k_sum_parts(int n, const double *part, double scale, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < n; ++i) t += part[i];
        *out = t * scale;
    }
}

// Adam on the FP32 master parameters, refreshed bfloat16 copies of the weights
__global__ void k_adam(long long n, float *w, const float *g, float *m, float *v, float lr,
                       float b1, float b2, float eps, float c1, float c2, __nv_bfloat16 *wb)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
}

__global__ void k_to_bf16(long long n, const float *w, __nv_bfloat16 *wb)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) wb[i] = __float2bfloat16_rn(w[i]);
}

// Fallback rule: for every patch, K_m = B + E + tr(B) sinh(out_m) / YS (E the
// resummed series estimate); flag when
//   max(max_{m,c} |K_m,c - mean_m K_m,c|, GAP_WEIGHT * gap) > thr * ||mean K||_F,
// gap = max_c |[4/4]_c - [3/3]_c| (how far the resummation is from converged).
// Surrogate estimate where not flagged: K = mean_m K_m.
__global__ void k_disagree(long long P, int members, const float *out, const double *B,
                           const double *E, double thr, double *K, int *flag)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const double tr = (B[3 * p] + B[3 * p + 2]) / MLSD_SUR_Y_SCALE;
    double mean[3] = {0, 0, 0};
    for (int m = 0; m < members; ++m)
        for (int c = 0; c < 3; ++c) mean[c] += sinh((double)out[((long long)m * P + p) * 3 + c]);
    double Km[3];
    for (int c = 0; c < 3; ++c) Km[c] = B[3 * p + c] + E[4 * p + c] + tr * mean[c] / members;
    const double fro = sqrt(Km[0] * Km[0] + 2.0 * Km[1] * Km[1] + Km[2] * Km[2]);
    double dev = MLSD_SUR_GAP_WEIGHT * E[4 * p + 3];
    for (int m = 0; m < members; ++m)
        for (int c = 0; c < 3; ++c) {
            const double km = B[3 * p + c] + E[4 * p + c]
                              + tr * sinh((double)out[((long long)m * P + p) * 3 + c]);
            dev = fmax(dev, fabs(km - Km[c]));
        }
    const int f = !(dev <= thr * fro);           // NaN -> flagged
    flag[p] = f;
    K[3 * p] = Km[0]; K[3 * p + 1] = Km[1]; K[3 * p + 2] = Km[2];
}

// Stable compaction of the flagged patch indices, one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_compact(long long P, const int *flag, int *idx, int *count)
{
    __shared__ int wsum[32];
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (long long c0 = 0; c0 < P; c0 += 1024) {
        const long long p = c0 + threadIdx.x;
        const int f = (p < P) ? flag[p] : 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        const int pre = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) wsum[w] = __popc(bal);
        __syncthreads();
        int off = 0;
        for (int q = 0; q < w; ++q) off += wsum[q];
        if (f) idx[base + off + pre] = (int)p;
        __syncthreads();
        if (threadIdx.x == 0) { int t = 0; for (int q = 0; q < 32; ++q) t += wsum[q]; base += t; }
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base;
}

// rows idx[0..M) of (X, Y) into the batch buffers (Xb, Yb)
// Source column and sign of column c of a feature row's image under symmetry g
// of the square (bit 0: reflect x1, bit 1: reflect x2, bit 2: then swap x1 and
// x2).  A reflection or a swap negates psi, so DFT entry (k1, k2) of the image
// is -1 per set bit times entry (k1s, k2s) of the source; symmetric tensors
// map as R T R^T.
__device__ __forceinline__ int sym_source(int c, int g, bool &neg)
{
    const bool rx = g & 1, ry = g & 2, sw = g & 4;
    neg = false;
    if (c < 2 * NMODE * NMODE) {
        const int m = c >> 1, k1 = m % NMODE - KMODE, k2 = m / NMODE - KMODE;
        const int q1 = sw ? k2 : k1, q2 = sw ? k1 : k2;
        const int k1s = rx ? -q1 : q1, k2s = ry ? -q2 : q2;
        neg = (rx != ry) != sw;
        return 2 * ((k2s + KMODE) * NMODE + (k1s + KMODE)) + (c & 1);
    }
    // B / kappa at 578..580, log kappa at 581, eight tensors at 582..605 (T_2..T_6
    // and the three approximants, each stored through the odd asinh), padding after
    const int base = c >= 582 && c < MLSD_SUR_FEATURES ? 582 + 3 * ((c - 582) / 3)
                                                       : (c >= 578 && c < 581 ? 578 : -1);
    if (base < 0) return c;
    const int i = c - base;
    if (i == 1) { neg = rx != ry; return c; }
    return sw ? base + 2 - i : c;
}

__device__ __forceinline__ float sym_target(const float *y, int i, int g)
{
    const bool rx = g & 1, ry = g & 2, sw = g & 4;
    if (i == 1) return rx != ry ? -y[1] : y[1];
    return sw ? y[2 - i] : y[i];
}

// Batch rows r < M: row idx[r] of (X, Y), or with aug its image under symmetry
// idx[r] & 7 of row idx[r] >> 3.  One CTA per row.
__global__ void k_gather_rows(int M, const int *idx, const __nv_bfloat16 *X, const float *Y,
                              __nv_bfloat16 *Xb, float *Yb, int aug)
{
    const int r = blockIdx.x;
    if (r >= M) return;
    const int v = idx[r];
    const long long src = aug ? v >> 3 : v;
    const int g = aug ? v & 7 : 0;
    if (g == 0) {
        const uint4 *xs = reinterpret_cast<const uint4 *>(X + src * MLSD_SUR_IN);
        uint4 *xd = reinterpret_cast<uint4 *>(Xb + (long long)r * MLSD_SUR_IN);
        for (int c = threadIdx.x; c < MLSD_SUR_IN / 8; c += blockDim.x) xd[c] = xs[c];
        if (threadIdx.x < 3) Yb[3 * r + threadIdx.x] = Y[3 * src + threadIdx.x];
        return;
    }
    const unsigned short *xs = reinterpret_cast<const unsigned short *>(X) + src * MLSD_SUR_IN;
    unsigned short *xd = reinterpret_cast<unsigned short *>(Xb) + (long long)r * MLSD_SUR_IN;
    for (int c = threadIdx.x; c < MLSD_SUR_IN; c += blockDim.x) {
        bool neg;
        const int sc = sym_source(c, g, neg);
        xd[c] = xs[sc] ^ (neg ? 0x8000u : 0u);          // bfloat16 negation: the sign bit
    }
    if (threadIdx.x < 3) Yb[3 * r + threadIdx.x] = sym_target(Y + 3 * src, threadIdx.x, g);
}

// image under symmetry g of rows r < n (either part skipped when its output is null)
__global__ void k_symmetry(long long n, int g, const __nv_bfloat16 *X, const float *Y,
                           __nv_bfloat16 *Xo, float *Yo)
{
    for (long long r = blockIdx.x; r < n; r += gridDim.x) {
        if (Xo) {
            const unsigned short *xs = reinterpret_cast<const unsigned short *>(X) + r * MLSD_SUR_IN;
            unsigned short *xd = reinterpret_cast<unsigned short *>(Xo) + r * MLSD_SUR_IN;
            for (int c = threadIdx.x; c < MLSD_SUR_IN; c += blockDim.x) {
                bool neg;
                const int sc = sym_source(c, g, neg);
                xd[c] = xs[sc] ^ (neg ? 0x8000u : 0u);
            }
        }
        if (Yo && threadIdx.x < 3) Yo[3 * r + threadIdx.x] = sym_target(Y + 3 * r, threadIdx.x, g);
    }
}

__global__ void k_add_loss(const double *loss, double *acc)
{
    if (threadIdx.x == 0) *acc += *loss;
}

// training targets asinh((K - B - E) YS / tr(B)) of one plain-solved level
// (E: the resummed series estimate, [P][4] with the series gap in the 4th column)
__global__ void k_targets(long long P, const double *B, const double *K, const double *E, float *Y)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const double f = MLSD_SUR_Y_SCALE / (B[3 * p] + B[3 * p + 2]);
    for (int c = 0; c < 3; ++c)
        Y[3 * p + c] = (float)asinh((K[3 * p + c] - B[3 * p + c] - E[4 * p + c]) * f);
}

// flagged patches take the plain solve: K = sym(B e_j + S_.j); with n_dev the
// count is read on the device (a launch sized for every patch)
__global__ void k_merge_fallback(int n, const int *n_dev, const int *idx, const double *B,
                                 const double *S, double *K)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (n_dev ? *n_dev : n)) return;
    const long long p = idx[t];
    const double *b = B + 3 * p, *s = S + 4 * p;
    K[3 * p] = b[0] + s[0];
    K[3 * p + 1] = 0.5 * ((b[1] + s[1]) + (b[1] + s[2]));
    K[3 * p + 2] = b[2] + s[3];
}

// Transpose of a row-major bfloat16 [rows][cols] (row stride cols) into [cols][ldT]:
// dst[c][r] = src[r][c] for r < rows, zero for rows <= r < ldT.  32 x 32 tiles
// through shared memory (reads and writes along rows).
__global__ void k_transpose_bf16(int rows, int cols, const __nv_bfloat16 *src, __nv_bfloat16 *dst,
                                 int ldT)
{
    __shared__ __nv_bfloat16 t[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        t[k][threadIdx.x] = (r < rows && c < cols) ? src[(long long)r * cols + c]
                                                   : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (c < cols && r < ldT) dst[(long long)c * ldT + r] = t[threadIdx.x][k];
    }
}

// Output layer of the tensor-core training step (3 outputs: one warp per row).
// Z4[m][j] = b4[j] + sum_k A3[m][k] W4[j][k]
__global__ void k_out_fwd(int M, int h, const __nv_bfloat16 *A3, const __nv_bfloat16 *W4,
                          const float *b4, float *Z4)
{
    const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (m >= M) return;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int k = lane; k < h; k += 32) {
        const float x = __bfloat162float(A3[(long long)m * h + k]);
        s0 = fmaf(x, __bfloat162float(W4[k]), s0);
        s1 = fmaf(x, __bfloat162float(W4[h + k]), s1);
        s2 = fmaf(x, __bfloat162float(W4[2 * h + k]), s2);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
        Z4[3 * m] = b4[0] + s0;
        Z4[3 * m + 1] = b4[1] + s1;
        Z4[3 * m + 2] = b4[2] + s2;
    }
}

// Partial sums of dW4[j][k] = sum_m dZ4[m][j] A3[m][k] and db4[j] = sum_m dZ4[m][j] over
// the row chunk blockIdx.y (rows y*chunk .. +chunk-1): a block of 32 columns x 8 row groups
// (rows g, g + 8, ...), reduced over the groups in order, into part[y][j][k] and (the
// blocks of the first column tile) bpart[y][j]; k_split_reduce adds the chunks in order
__global__ void k_out_bwd_w(int M, int h, int chunk, const float *dZ4, const __nv_bfloat16 *A3,
                            float *part, float *bpart)
{
    __shared__ float red[8][4][33];
    const int c = threadIdx.x & 31, g = threadIdx.x >> 5, k = blockIdx.x * 32 + c;
    const int mb = blockIdx.y * chunk, me = min(M, mb + chunk);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, b = 0.f;
    for (int m = mb + g; m < me; m += 8) {
        const float x = k < h ? __bfloat162float(A3[(long long)m * h + k]) : 0.f;
        const float d0 = dZ4[3 * m], d1 = dZ4[3 * m + 1], d2 = dZ4[3 * m + 2];
        s0 = fmaf(d0, x, s0);
        s1 = fmaf(d1, x, s1);
        s2 = fmaf(d2, x, s2);
        if (c < 3) b += c == 0 ? d0 : (c == 1 ? d1 : d2);
    }
    red[g][0][c] = s0; red[g][1][c] = s1; red[g][2][c] = s2; red[g][3][c] = b;
    __syncthreads();
    if (g < 3 && k < h) {
        float t = 0.f;
        for (int q = 0; q < 8; ++q) t += red[q][g][c];
        part[((long long)blockIdx.y * 3 + g) * h + k] = t;
    }
    if (blockIdx.x == 0 && g == 3 && c < 3) {
        float t = 0.f;
        for (int q = 0; q < 8; ++q) t += red[q][3][c];
        bpart[blockIdx.y * 3 + c] = t;
    }
}

// dZ3 = bf16((dZ4 W4) gelu'(Z3)) into bfloat16 [M][h] and its transpose [h][ldT] (zero
// for M <= m < ldT): 32 x 32 tiles through shared memory
__global__ void k_out_bwd_x(int M, int h, const float *dZ4, const __nv_bfloat16 *W4, const float *Z3,
                            __nv_bfloat16 *dZ, __nv_bfloat16 *dZT, int ldT)
{
    __shared__ __nv_bfloat16 t[32][33];
    const int m0 = blockIdx.y * 32, k0 = blockIdx.x * 32, k = k0 + threadIdx.x;
    float w0 = 0.f, w1 = 0.f, w2 = 0.f;
    if (k < h) {
        w0 = __bfloat162float(W4[k]); w1 = __bfloat162float(W4[h + k]); w2 = __bfloat162float(W4[2 * h + k]);
    }
    for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        const int m = m0 + q;
        __nv_bfloat16 v = __float2bfloat16_rn(0.f);
        if (m < M && k < h) {
            float d = dZ4[3 * m] * w0;
            d = fmaf(dZ4[3 * m + 1], w1, d);
            d = fmaf(dZ4[3 * m + 2], w2, d);
            v = __float2bfloat16_rn(d * gelu_d(Z3[(long long)m * h + k]));
            dZ[(long long)m * h + k] = v;
        }
        t[q][threadIdx.x] = v;
    }
    __syncthreads();
    for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        const int kk = k0 + q, m = m0 + threadIdx.x;
        if (kk < h && m < ldT) dZT[(long long)kk * ldT + m] = t[threadIdx.x][q];
    }
}

// FP32 [M][N] (bfloat16-valued) to bfloat16 [M][N] and its transpose [N][ldT] (zero for
// M <= m < ldT)
__global__ void k_to_bf16_t(int M, int N, const float *src, __nv_bfloat16 *dst, __nv_bfloat16 *dstT,
                            int ldT)
{
    __shared__ __nv_bfloat16 t[32][33];
    const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int m = m0 + k, n = n0 + threadIdx.x;
        __nv_bfloat16 v = __float2bfloat16_rn(0.f);
        if (m < M && n < N) {
            v = __float2bfloat16_rn(src[(long long)m * N + n]);
            dst[(long long)m * N + n] = v;
        }
        t[k][threadIdx.x] = v;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int n = n0 + k, m = m0 + threadIdx.x;
        if (n < N && m < ldT) dstT[(long long)n * ldT + m] = t[threadIdx.x][k];
    }
}

// out[r] = sum over k < K of src[r][k] (bfloat16, row stride ld a multiple of 8, zero
// padding up to ld), one warp per row, FP32 in a fixed order (each lane sums 16-byte
// vectors 8 k apart, then the warp tree)
__global__ void k_rowsum_bf16(int rows, int K, const __nv_bfloat16 *src, int ld, float *out)
{
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r >= rows) return;
    float acc = 0.f;
    const __nv_bfloat16 *row = src + (long long)r * ld;
    for (int k = 8 * lane; k < K; k += 256) {
        const uint4 q = *reinterpret_cast<const uint4 *>(row + k);
        const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&q);
#pragma unroll
        for (int i = 0; i < 8; ++i) acc += __bfloat162float(e[i]);   // zeros past K
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[r] = acc;
}

}  // namespace

// ---------------------------------------------------------------------------
// Host-side pieces used by the runtime
long long sur_param_count(int h)
{
    return (long long)h * MLSD_SUR_IN + h + 2 * ((long long)h * h + h) + 3LL * h + 3;
}

template <int N>
static cudaError_t launch_series(const float *band, long long Nl, long long tile, int n, int sub,
                                 int n_macro, const int *pidx, long long count, const double *B,
                                 void *X, float *F32, double *E, cudaStream_t s)
{
    const size_t smem = (size_t)N * N * (8 + 5 * 4) + (size_t)N / 2 * 8;
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(&k_series<N>),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_series<N><<<(unsigned)count, 256, smem, s>>>(band, Nl, tile, n, sub, n_macro, pidx, count,
                                                   B, static_cast<__nv_bfloat16 *>(X), F32, E);
    return cudaGetLastError();
}

// Features of n x n patches, n = 32, 64, 128 or 256: patches above 64 x 64 are
// described by their samples on the 64 x 64 sub-lattice (every n/64-th node)
cudaError_t launch_features(const float *band, long long Nl, long long tile, int n, int n_macro,
                            const int *pidx, long long count, const double *B, double kappa,
                            void *X, float *F32, double *E, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    if (n != 32 && n != 64 && n != 128 && n != 256) return cudaErrorInvalidValue;
    const int nf = n < 64 ? n : 64, sub = n / nf;
    const size_t smem = (size_t)nf * nf * 4 + (size_t)nf * NMODE * 8;
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(&k_features),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_features<<<(unsigned)count, 320, smem, s>>>(band, Nl, tile, n, sub, n_macro, pidx, count, B,
                                                  kappa, static_cast<__nv_bfloat16 *>(X), F32);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return nf == 32 ? launch_series<32>(band, Nl, tile, n, sub, n_macro, pidx, count, B, X, F32, E, s)
                    : launch_series<64>(band, Nl, tile, n, sub, n_macro, pidx, count, B, X, F32, E, s);
}

template <int N>
static cudaError_t launch_periodize_n(const float *band, long long Nl, int n_macro, const int *pidx,
                                      long long count, float *tiles, cudaStream_t s)
{
    const size_t smem = (size_t)N * N * 12 + (size_t)N / 2 * 8;
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(&k_periodize<N>),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_periodize<N><<<(unsigned)count, 256, smem, s>>>(band, Nl, n_macro, pidx, count, tiles);
    return cudaGetLastError();
}

cudaError_t launch_periodize(const float *band, long long Nl, int n, int n_macro, const int *pidx,
                             long long count, float *tiles, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    if (n == 32) return launch_periodize_n<32>(band, Nl, n_macro, pidx, count, tiles, s);
    if (n == 64) return launch_periodize_n<64>(band, Nl, n_macro, pidx, count, tiles, s);
    return cudaErrorInvalidValue;
}

// Layer views of one member's parameters (FP32 master or bfloat16 copy)
struct Layers {
    long long w[4], b[4];
    int din[4], dout[4];
};
static Layers layers(int h)
{
    Layers L;
    const int dims[5] = {MLSD_SUR_IN, h, h, h, 3};
    long long o = 0;
    for (int l = 0; l < 4; ++l) {
        L.din[l] = dims[l];
        L.dout[l] = dims[l + 1];
        L.w[l] = o; o += (long long)dims[l + 1] * dims[l];
        L.b[l] = o; o += dims[l + 1];
    }
    return L;
}

// Forward of one member on M rows: Z_l (FP32) and bf16 activations A_l.
// ws: Z1..Z3 [M][h], Z4 [M][3] FP32; A1..A3 [M][h] bf16.
cudaError_t sur_forward(int h, int M, const void *X, const float *wf, const void *wb_,
                        float *Z[4], void *Aact[3], float *ws, long long ws_n, cudaStream_t s)
{
    const Layers L = layers(h);
    const __nv_bfloat16 *wb = static_cast<const __nv_bfloat16 *>(wb_);
    const __nv_bfloat16 *in = static_cast<const __nv_bfloat16 *>(X);
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
        Epi ep;
        ep.bias = wf + L.b[l];
        ep.act = l < 3 ? static_cast<__nv_bfloat16 *>(Aact[l]) : nullptr;
        ep.sactm = L.dout[l];
        e = gemm<__nv_bfloat16, __nv_bfloat16>(s, M, L.dout[l], L.din[l], in, L.din[l], 1,
                                               wb + L.w[l], 1, L.din[l], Z[l], L.dout[l], ep, ws,
                                               ws_n);
        in = ep.act;
    }
    return e;
}

long long sur_split_workspace(int h) { return (long long)SPLIT_MAX * h * (MLSD_SUR_IN + 1); }

cudaError_t sur_grad(int h, int M, const void *X, const float *Y, const float *wf, const void *wb_,
                     float *Z[4], void *Aact[3], float *dA, float *dB_, float *g, double *part,
                     double *loss_dev, float *ws, long long ws_n, cudaStream_t s)
{
    const Layers L = layers(h);
    const __nv_bfloat16 *wb = static_cast<const __nv_bfloat16 *>(wb_);
    cudaError_t e = sur_forward(h, M, X, wf, wb_, Z, Aact, ws, ws_n, s);
    if (e != cudaSuccess) return e;
    const int nb = (3 * M + 255) / 256;
    count_launches(2);
    k_mse<<<nb, 256, 0, s>>>(M, Z[3], Y, dA, part);
    k_sum_parts<<<1, 32, 0, s>>>(nb, part, 1.0 / (3.0 * M), loss_dev);
    float *dZ = dA, *dN = dB_;
    for (int l = 3; l >= 0; --l) {
        const __nv_bfloat16 *Ain = l > 0 ? static_cast<const __nv_bfloat16 *>(Aact[l - 1])
                                         : static_cast<const __nv_bfloat16 *>(X);
        // dW_l[j][k] = sum_m dZ[m][j] Ain[m][k], and the bias gradient db_l[j] = sum_m dZ[m][j]
        // as the row sums of the same GEMM's A operand
        e = gemm<float, __nv_bfloat16>(s, L.dout[l], L.din[l], M, dZ, 1, L.dout[l], Ain, L.din[l],
                                       1, g + L.w[l], L.din[l], Epi{}, ws, ws_n, g + L.b[l]);
        if (e != cudaSuccess) return e;
        if (l == 0) break;
        // dZ_{l-1}[m][k] = (sum_j dZ[m][j] W_l[j][k]) gelu'(Z_{l-1}[m][k])
        Epi ep;
        ep.dgelu = Z[l - 1];
        e = gemm<float, __nv_bfloat16>(s, M, L.din[l], L.dout[l], dZ, L.dout[l], 1, wb + L.w[l],
                                       L.din[l], 1, dN, L.din[l], ep, ws, ws_n);
        if (e != cudaSuccess) return e;
        float *t = dZ; dZ = dN; dN = t;
    }
    return cudaGetLastError();
}

// The gradient of one member with the hidden layers' contractions on the tensor cores
// (gemm_tc): forward Z_l = A_{l-1} W_l^T + b_l with bfloat16 act_l and its transpose,
// l = 0..2; the output layer, the loss and the output layer's gradients as in sur_grad
// (CUDA cores); then for l = 2, 1, 0: dW_l = dZ_l^T A_{l-1} (K = the batch, split over
// CTAs, partials summed in a fixed order), db_l = the row sums of dZ_l^T, and
// dZ_{l-1} = bf16((dZ_l W_l) gelu'(Z_{l-1})) and its transpose.  dZ of the hidden
// layers is a bfloat16 operand throughout (the oracle's emulation rounds it the same).
cudaError_t sur_grad_tc(int h, int M, const void *X, const float *Y, const float *wf,
                        const void *wb_, float *Z[4], void *Aact[3], float *dA, float *dB_,
                        float *g, double *part, double *loss_dev, float *ws, long long ws_n,
                        const SurTc &tc, int *status, cudaStream_t s)
{
    const Layers L = layers(h);
    const __nv_bfloat16 *wb = static_cast<const __nv_bfloat16 *>(wb_);
    const int ldT = tc.ldT;
    if (M > tc.max_rows || ldT < ((M + 7) / 8) * 8) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    const dim3 tb(32, 8);
    auto tgrid = [](int rows, int cols) { return dim3((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32)); };
    // W_1^T, W_2^T for the data gradients
    count_launches(2);
    for (int l = 1; l <= 2; ++l)
        k_transpose_bf16<<<tgrid(h, h), tb, 0, s>>>(h, h, wb + L.w[l], tc.WT[l - 1], h);
    e = cudaGetLastError();
    // forward, hidden layers on the tensor cores
    const __nv_bfloat16 *in = static_cast<const __nv_bfloat16 *>(X);
    for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
        e = gemm_tc(0, M, h, L.din[l], in, L.din[l], wb + L.w[l], L.din[l], wf + L.b[l], Z[l],
                    nullptr, Aact[l], tc.AT[l], ldT, nullptr, 1, nullptr, status, s);
        in = static_cast<const __nv_bfloat16 *>(Aact[l]);
    }
    if (e != cudaSuccess) return e;
    // output layer (3 outputs) and its gradients, on the CUDA cores: Z4, the loss and
    // dZ4, dW4 and db4, and dZ3 = bf16((dZ4 W4) gelu'(Z3)) with its transpose
    const int nb = (3 * M + 255) / 256;
    count_launches(6);
    k_out_fwd<<<(unsigned)((M + 7) / 8), 256, 0, s>>>(M, h, in, wb + L.w[3], wf + L.b[3], Z[3]);
    k_mse<<<nb, 256, 0, s>>>(M, Z[3], Y, dA, part);
    k_sum_parts<<<1, 32, 0, s>>>(nb, part, 1.0 / (3.0 * M), loss_dev);
    {
        const int S = std::min(16, (M + 127) / 128), chunk = (M + S - 1) / S;
        float *bpart = ws + (long long)S * 3 * h;
        k_out_bwd_w<<<dim3((unsigned)((h + 31) / 32), (unsigned)S), 256, 0, s>>>(M, h, chunk, dA, in,
                                                                              ws, bpart);
        count_launches(1);
        k_split_reduce<<<(unsigned)((3 * h + 3 + 255) / 256), 256, 0, s>>>(3, h, S, ws, g + L.w[3], h,
                                                                          Epi{}, bpart, g + L.b[3]);
    }
    k_out_bwd_x<<<tgrid(M, h), tb, 0, s>>>(M, h, dA, wb + L.w[3], Z[2], tc.dZ[0], tc.dZT[0], ldT);
    k_transpose_bf16<<<tgrid(M, MLSD_SUR_IN), tb, 0, s>>>(M, MLSD_SUR_IN, static_cast<const __nv_bfloat16 *>(X),
                                                         tc.XT, ldT);
    e = cudaGetLastError();
    (void)dB_;
    int cur = 0;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int l = 2; l >= 0 && e == cudaSuccess; --l) {
        const int din = L.din[l];
        const void *Bt = l > 0 ? static_cast<const void *>(tc.AT[l - 1]) : static_cast<const void *>(tc.XT);
        // dW_l[j][k] = sum_m dZ[m][j] A_{l-1}[m][k]: A = dZ^T [h][M], B = A_{l-1}^T [din][M]
        int splits = gemm_tc_splits(h, din, M, sms);
        while (splits > 1 && (long long)splits * h * din > ws_n) --splits;
        int used = 1;
        e = gemm_tc(2, h, din, M, tc.dZT[cur], ldT, Bt, ldT, nullptr, nullptr, nullptr, nullptr,
                    nullptr, ldT, ws, splits, &used, status, s);
        if (e != cudaSuccess) break;
        const long long n = (long long)h * din;
        count_launches(2);
        k_split_reduce<<<(unsigned)std::min<long long>((n + 255) / 256, 8LL * sms), 256, 0, s>>>(
            h, din, used, ws, g + L.w[l], din, Epi{}, nullptr, nullptr);
        k_rowsum_bf16<<<(unsigned)((h + 7) / 8), 256, 0, s>>>(h, M, tc.dZT[cur], ldT, g + L.b[l]);
        e = cudaGetLastError();
        if (e != cudaSuccess || l == 0) break;
        // dZ_{l-1} = bf16((dZ_l W_l) gelu'(Z_{l-1})): A = dZ_l [M][h], B = W_l^T [din][h]
        e = gemm_tc(1, M, din, h, tc.dZ[cur], h, tc.WT[l - 1], h, nullptr, nullptr, Z[l - 1],
                    tc.dZ[cur ^ 1], tc.dZT[cur ^ 1], ldT, nullptr, 1, nullptr, status, s);
        cur ^= 1;
    }
    return e;
}

cudaError_t sur_adam(long long n, float *w, const float *g, float *m, float *v, float lr, int t,
                     void *wb, cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    count_launches(1);
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, w, g, m, v, lr, b1, b2, 1e-8f, c1, c2,
                                                      static_cast<__nv_bfloat16 *>(wb));
    return cudaGetLastError();
}

cudaError_t sur_to_bf16(long long n, const float *w, void *wb, cudaStream_t s)
{
    count_launches(1);
    k_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, w, static_cast<__nv_bfloat16 *>(wb));
    return cudaGetLastError();
}

cudaError_t sur_gather(int M, const int *idx, const void *X, const float *Y, void *Xb, float *Yb,
                       int aug, cudaStream_t s)
{
    count_launches(1);
    k_gather_rows<<<(unsigned)M, 128, 0, s>>>(M, idx, static_cast<const __nv_bfloat16 *>(X), Y,
                                              static_cast<__nv_bfloat16 *>(Xb), Yb, aug);
    return cudaGetLastError();
}

cudaError_t sur_symmetry(long long n, int g, const void *X, const float *Y, void *Xo, float *Yo,
                         cudaStream_t s)
{
    if (n < 1) return cudaSuccess;
    count_launches(1);
    const unsigned nb = (unsigned)std::min<long long>(n, 65535LL * 16);
    k_symmetry<<<nb, 128, 0, s>>>(n, g, static_cast<const __nv_bfloat16 *>(X), Y,
                                  static_cast<__nv_bfloat16 *>(Xo), Yo);
    return cudaGetLastError();
}

cudaError_t sur_add_loss(const double *loss, double *acc, cudaStream_t s)
{
    count_launches(1);
    k_add_loss<<<1, 32, 0, s>>>(loss, acc);
    return cudaGetLastError();
}

cudaError_t sur_targets(long long P, const double *B, const double *K, const double *E, float *Y,
                        cudaStream_t s)
{
    count_launches(1);
    k_targets<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(P, B, K, E, Y);
    return cudaGetLastError();
}

cudaError_t sur_disagree(long long P, int members, const float *out, const double *B,
                         const double *E, double thr, double *K, int *flag, int *idx, int *count,
                         cudaStream_t s)
{
    count_launches(2);
    k_disagree<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(P, members, out, B, E, thr, K, flag);
    k_compact<<<1, 1024, 0, s>>>(P, flag, idx, count);
    return cudaGetLastError();
}

cudaError_t sur_merge(int n, const int *idx, const double *B, const double *S, double *K,
                      cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    count_launches(1);
    k_merge_fallback<<<(n + 255) / 256, 256, 0, s>>>(n, nullptr, idx, B, S, K);
    return cudaGetLastError();
}

cudaError_t sur_merge_dev(long long P, const int *n_dev, const int *idx, const double *B,
                          const double *S, double *K, cudaStream_t s)
{
    count_launches(1);
    k_merge_fallback<<<(unsigned)((P + 255) / 256), 256, 0, s>>>((int)P, n_dev, idx, B, S, K);
    return cudaGetLastError();
}

}  // namespace mlsd
