// Level hierarchy on the device: band synthesis (Sec. 3.1), the line
// variances and harmonic means of Algorithms 1-2, and the per-patch tensor
// bookkeeping of Algorithm 3.
#include "mlsd_internal.cuh"

namespace mlsd {
namespace {

// cos/sin(2 pi r / Nl) for an exactly reduced phase index r in [0, Nl)
__device__ __forceinline__ void twiddle(long long r, long long Nl, double &c, double &s)
{
    sincospi(2.0 * (double)r / (double)Nl, &s, &c);
}

// Pass 1: G[g][y] = sum_{modes of group g} (re + i im) e^{i k2 2 pi y / Nl}
__global__ void k_band_pass1(ModeGroups m, long long Nl, double2 *G)
{
    const int g = blockIdx.y;
    const long long y = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (y >= Nl) return;
    double gr = 0.0, gi = 0.0;
    for (int t = m.gofs[g]; t < m.gofs[g + 1]; ++t) {
        double c, s;
        twiddle(pmod_ll((long long)m.k2[t] * y, Nl), Nl, c, s);
        const double re = m.re[t], im = m.im[t];
        gr += re * c - im * s;
        gi += re * s + im * c;
    }
    G[(long long)g * Nl + y] = make_double2(gr, gi);
}

// Pass 2: psi[y][x] = sum_g Re(e^{i k1_g 2 pi x / Nl} G[g][y])
template <typename T>
__global__ void k_band_pass2(ModeGroups m, long long Nl, const double2 *G, T *out)
{
    const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long y = blockIdx.y;
    if (x >= Nl) return;
    double acc = 0.0;
    for (int g = 0; g < m.n_groups; ++g) {
        double c, s;
        twiddle(pmod_ll((long long)m.gk1[g] * x, Nl), Nl, c, s);
        const double2 v = G[(long long)g * Nl + y];
        acc += v.x * c - v.y * s;
    }
    out[y * Nl + x] = (T)acc;
}

// Factorised Algorithm 1 line variances.  An off-diagonal part restricted to a
// patch line (psi_12 on a column x = x_a, psi_21 on a row y = y_b) is
//   g(s) = Re sum_groups e^{i kc x_line} G_o(kc, s),
//   G_o(kc, s) = sum_{modes with that kc} c e^{i kv t_s},
// where kc is the wavenumber across the line (k1 for psi_12) and kv the one
// along it; the samples t_s of every patch of macro row (column) o coincide,
// so G is synthesised once per o (pass A) and combined per patch line (pass B).
//   Gout[o][g][s], o < n_macro, g < groups, s < ms (samples per line)
__global__ void k_line_synth(ModeGroups grp, long long Nl, int n, int r, int n_macro, int ms,
                             double2 *Gout)
{
    const int o = blockIdx.y, g = blockIdx.z;
    const long long Nr = Nl * r;
    const long long t0 = patch_origin(o, n_macro, Nl, n) * r;     // first sample's lattice index
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < ms; s += gridDim.x * blockDim.x) {
        double gr = 0.0, gi = 0.0;
        for (int t = grp.gofs[g]; t < grp.gofs[g + 1]; ++t) {
            double c, sn;
            twiddle(pmod_ll((long long)grp.k2[t] * (t0 + s), Nr), Nr, c, sn);
            gr += grp.re[t] * c - grp.im[t] * sn;
            gi += grp.re[t] * sn + grp.im[t] * c;
        }
        Gout[((long long)o * grp.n_groups + g) * ms + s] = make_double2(gr, gi);
    }
}

// one CTA per (patch, line): variance over the ms samples of the line
__global__ void k_line_var(ModeGroups grp, const double2 *G, long long Nl, int n, int ms,
                           int n_macro, int along_x2, const int *idx, int stride, double *q)
{
    __shared__ double red[2][32];
    __shared__ double2 tw[256];
    const long long p = idx ? (long long)idx[blockIdx.x] : (long long)blockIdx.x;
    const int line = blockIdx.y;
    // psi_12 (along x2): line origin o = macro row, constant coordinate = column x_a;
    // psi_21 (along x1): o = macro column, constant coordinate = row y_b
    const long long o = along_x2 ? p / n_macro : p % n_macro;
    const long long oc = patch_origin(along_x2 ? p % n_macro : p / n_macro, n_macro, Nl, n);
    for (int g = threadIdx.x; g < grp.n_groups; g += blockDim.x) {
        double c, sn;
        twiddle(pmod_ll((long long)grp.gk1[g] * (oc + line), Nl), Nl, c, sn);
        tw[g] = make_double2(c, sn);
    }
    __syncthreads();
    const double2 *Go = G + o * grp.n_groups * (long long)ms;
    double ref = 0.0;
    for (int g = 0; g < grp.n_groups; ++g) ref += Go[(long long)g * ms].x * tw[g].x - Go[(long long)g * ms].y * tw[g].y;
    double s1 = 0.0, s2 = 0.0;
    for (int s = threadIdx.x; s < ms; s += blockDim.x) {
        double v = 0.0;
        for (int g = 0; g < grp.n_groups; ++g) {
            const double2 a = Go[(long long)g * ms + s];
            v += a.x * tw[g].x - a.y * tw[g].y;
        }
        v -= ref;
        s1 += v;
        s2 += v * v;
    }
    for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = s1; red[1][threadIdx.x >> 5] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red[0][w]; b += red[1][w]; }
        const double mean = a / (double)ms;
        const double var = b / (double)ms - mean * mean;
        q[p * stride + line] = var > 0.0 ? var : 0.0;
    }
}

// per patch: max over its nref x nref reference nodes of sqrt(v1^2 + v2^2)
__global__ void k_patch_vmax(const double *v1, const double *v2, long long Nr, int nref,
                             int n_macro, double *vmax)
{
    __shared__ double red[32];
    const long long p = blockIdx.x;
    const long long ox = patch_origin(p % n_macro, n_macro, Nr, nref);
    const long long oy = patch_origin(p / n_macro, n_macro, Nr, nref);
    double m = 0.0;
    for (int c = threadIdx.x; c < nref * nref; c += blockDim.x) {
        const long long gy = pmod_ll(oy + c / nref, Nr), gx = pmod_ll(ox + c % nref, Nr);
        const double a = v1[gy * Nr + gx], b = v2[gy * Nr + gx];
        m = fmax(m, sqrt(a * a + b * b));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
        vmax[p] = t;
    }
}

// Algorithms 1-2 for one patch: K_off = K[psi_12; B] + K[psi_21; B] - B with the
// shear closed forms K*11 = B11 + q12/B22, K*22 = B22 + q21/B11 on every line
// and their harmonic means.  A part that is absent leaves B unchanged.
__device__ void offdiag_apply(const OffdiagLevel &o, long long p, const double *B, double *K)
{
    double k12_11 = B[0], k21_22 = B[2];
    const int n = o.np ? o.np[p] : o.stride;
    if (o.q12) {
        double s = 0.0;
        for (int a = 0; a < n; ++a) s += 1.0 / (B[0] + o.q12[p * o.stride + a] / B[2]);
        k12_11 = (double)n / s;
    }
    if (o.q21) {
        double s = 0.0;
        for (int b = 0; b < n; ++b) s += 1.0 / (B[2] + o.q21[p * o.stride + b] / B[0]);
        k21_22 = (double)n / s;
    }
    if (!o.q12 && !o.q21) { K[0] = B[0]; K[1] = B[1]; K[2] = B[2]; return; }
    K[0] = k12_11 + B[0] - B[0];
    K[1] = B[1] + B[1] - B[1];
    K[2] = B[2] + k21_22 - B[2];
}

// Top-down closed forms: B_1 = kappa I, Koff_l = K_off,l(B_l), B_{l+1} = Koff_l.
__global__ void k_topdown(ChainTables t)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= t.P) return;
    double B[3] = {t.kappa, 0.0, t.kappa}, K[3];
    for (int l = 0; l < t.L; ++l) {
        t.B[l][3 * p] = B[0]; t.B[l][3 * p + 1] = B[1]; t.B[l][3 * p + 2] = B[2];
        offdiag_apply(t.off[l], p, B, K);
        t.Koff[l][3 * p] = K[0]; t.Koff[l][3 * p + 1] = K[1]; t.Koff[l][3 * p + 2] = K[2];
        B[0] = K[0]; B[1] = K[1]; B[2] = K[2];
    }
}

__global__ void k_level_base(long long P, int finest, const double *base_next, const double *S_next,
                             double *Kstar_next, const double *Koff_l, const double *B_l,
                             OffdiagLevel off, double *base_out)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    double X[3];
    if (finest) {
        X[0] = B_l[3 * p]; X[1] = B_l[3 * p + 1]; X[2] = B_l[3 * p + 2];
    } else {
        // K*_{l+1} = sym(P) with P_j = B e_j + S_.j  (same order as the compose step)
        const double *b = base_next + 3 * p, *s = S_next + 4 * p;
        const double k11 = b[0] + s[0], k12 = 0.5 * ((b[1] + s[1]) + (b[1] + s[2])), k22 = b[2] + s[3];
        if (Kstar_next) { Kstar_next[3 * p] = k11; Kstar_next[3 * p + 1] = k12; Kstar_next[3 * p + 2] = k22; }
        // Algorithm 3 step 3: K*_net = K* - K_off + B
        X[0] = k11 - Koff_l[3 * p] + B_l[3 * p];
        X[1] = k12 - Koff_l[3 * p + 1] + B_l[3 * p + 1];
        X[2] = k22 - Koff_l[3 * p + 2] + B_l[3 * p + 2];
    }
    double K[3];
    offdiag_apply(off, p, X, K);
    base_out[3 * p] = K[0]; base_out[3 * p + 1] = K[1]; base_out[3 * p + 2] = K[2];
}

// Energy form of the corrector pair of one patch (one CTA per patch, FP64 sums):
//   E_jk = < B11 D+x w_j D+x w_k + B12 (D0x w_j D0y w_k + D0y w_j D0x w_k) + B22 D+y w_j D+y w_k >
// and the means <w_j>.  Multiplying the steady corrector equation by w_k and
// summing by parts (D+D- against D+, D0 skew-adjoint) gives E = sym<v w> = K - B
// up to the O(h^2) remainder of the central advection term, which the grid does
// not make skew-adjoint (exact for shear flows).
template <typename real>
__global__ void __launch_bounds__(256) k_corrector_energy(int n, double h, const real *w, const double *B,
                                                          double *E, double *M)
{
    const long long p = blockIdx.x;
    const long long nn = (long long)n * n;
    const real *w1 = w + 2 * p * nn, *w2 = w1 + nn;
    const double B11 = B[3 * p], B12 = B[3 * p + 1], B22 = B[3 * p + 2];
    double acc[5] = {0, 0, 0, 0, 0};               // e11, e12, e22, m1, m2
    for (long long c = threadIdx.x; c < nn; c += blockDim.x) {
        const int a = (int)(c % n), b = (int)(c / n);
        const int ap = (a + 1) % n, am = (a + n - 1) % n, bp = (b + 1) % n, bm = (b + n - 1) % n;
        const double u1 = w1[c], u2 = w2[c];
        const double fx1 = (double)w1[(long long)b * n + ap] - u1, fy1 = (double)w1[(long long)bp * n + a] - u1;
        const double fx2 = (double)w2[(long long)b * n + ap] - u2, fy2 = (double)w2[(long long)bp * n + a] - u2;
        const double cx1 = 0.5 * ((double)w1[(long long)b * n + ap] - (double)w1[(long long)b * n + am]);
        const double cy1 = 0.5 * ((double)w1[(long long)bp * n + a] - (double)w1[(long long)bm * n + a]);
        const double cx2 = 0.5 * ((double)w2[(long long)b * n + ap] - (double)w2[(long long)b * n + am]);
        const double cy2 = 0.5 * ((double)w2[(long long)bp * n + a] - (double)w2[(long long)bm * n + a]);
        acc[0] += B11 * fx1 * fx1 + 2.0 * B12 * cx1 * cy1 + B22 * fy1 * fy1;
        acc[1] += B11 * fx1 * fx2 + B12 * (cx1 * cy2 + cy1 * cx2) + B22 * fy1 * fy2;
        acc[2] += B11 * fx2 * fx2 + 2.0 * B12 * cx2 * cy2 + B22 * fy2 * fy2;
        acc[3] += u1;
        acc[4] += u2;
    }
    __shared__ double red[5][8];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[threadIdx.x][k];
        if (threadIdx.x < 3) E[3 * p + threadIdx.x] = t / ((double)nn * h * h);
        else if (M) M[2 * p + threadIdx.x - 3] = t / (double)nn;
    }
}

// flux averages that reproduce a given K* on the base: S = K* - B (both off-diagonal
// entries carry K*12 - B12), as the chain reads a surrogate level
__global__ void k_S_from_K(long long P, const double *base, const double *K, double *S)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    S[4 * p] = K[3 * p] - base[3 * p];
    S[4 * p + 1] = S[4 * p + 2] = K[3 * p + 1] - base[3 * p + 1];
    S[4 * p + 3] = K[3 * p + 2] - base[3 * p + 2];
}

__global__ void k_offdiag_apply(long long P, OffdiagLevel off, const double *B, double *Koff)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    double X[3] = {B[3 * p], B[3 * p + 1], B[3 * p + 2]}, K[3];
    offdiag_apply(off, p, X, K);
    Koff[3 * p] = K[0]; Koff[3 * p + 1] = K[1]; Koff[3 * p + 2] = K[2];
}

}  // namespace

cudaError_t launch_band_synth(const ModeGroups &m, long long Nl, double2 *G, void *out,
                              int out_double, cudaStream_t s)
{
    if (m.n_groups == 0) {
        return cudaMemsetAsync(out, 0, (size_t)Nl * Nl * (out_double ? 8 : 4), s);
    }
    const int t = 256;
    dim3 g1((unsigned)((Nl + t - 1) / t), (unsigned)m.n_groups);
    count_launches(2);
    k_band_pass1<<<g1, t, 0, s>>>(m, Nl, G);
    dim3 g2((unsigned)((Nl + t - 1) / t), (unsigned)Nl);
    if (out_double) k_band_pass2<double><<<g2, t, 0, s>>>(m, Nl, G, static_cast<double *>(out));
    else k_band_pass2<float><<<g2, t, 0, s>>>(m, Nl, G, static_cast<float *>(out));
    return cudaGetLastError();
}

cudaError_t launch_line_var(const ModeGroups &grp, long long Nl, int n, int r, int n_macro,
                            long long count, const int *idx, int along_x2, int stride, double *q,
                            double2 *Gscratch, cudaStream_t s)
{
    if (grp.n_groups == 0 || count == 0) return cudaSuccess;
    if (grp.n_groups > 256) return cudaErrorInvalidValue;
    const int ms = n * r;
    dim3 ga((unsigned)((ms + 127) / 128), (unsigned)n_macro, (unsigned)grp.n_groups);
    count_launches(2);
    k_line_synth<<<ga, 128, 0, s>>>(grp, Nl, n, r, n_macro, ms, Gscratch);
    dim3 gb((unsigned)count, (unsigned)n);
    k_line_var<<<gb, 128, 0, s>>>(grp, Gscratch, Nl, n, ms, n_macro, along_x2, idx, stride, q);
    return cudaGetLastError();
}

cudaError_t launch_patch_vmax(const double *v1, const double *v2, long long Nr, int nref,
                              int n_macro, long long P, double *vmax, cudaStream_t s)
{
    count_launches(1);
    k_patch_vmax<<<(unsigned)P, 256, 0, s>>>(v1, v2, Nr, nref, n_macro, vmax);
    return cudaGetLastError();
}

cudaError_t launch_topdown(const ChainTables &t, cudaStream_t s)
{
    const int th = 128;
    count_launches(1);
    k_topdown<<<(unsigned)((t.P + th - 1) / th), th, 0, s>>>(t);
    return cudaGetLastError();
}

cudaError_t launch_level_base(long long P, int finest, const double *base_next,
                              const double *S_next, double *Kstar_next, const double *Koff_l,
                              const double *B_l, OffdiagLevel off, double *base_out,
                              cudaStream_t s)
{
    const int th = 128;
    count_launches(1);
    k_level_base<<<(unsigned)((P + th - 1) / th), th, 0, s>>>(P, finest, base_next, S_next,
                                                               Kstar_next, Koff_l, B_l, off,
                                                               base_out);
    return cudaGetLastError();
}

cudaError_t launch_S_from_K(long long P, const double *base, const double *K, double *S, cudaStream_t s)
{
    count_launches(1);
    k_S_from_K<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(P, base, K, S);
    return cudaGetLastError();
}

cudaError_t launch_corrector_energy(int n, double h, long long P, int precision, const void *w,
                                   const double *B, double *E, double *M, cudaStream_t s)
{
    if (P == 0) return cudaSuccess;
    count_launches(1);
    if (precision == MLSD_FP64)
        k_corrector_energy<double><<<(unsigned)P, 256, 0, s>>>(n, h, static_cast<const double *>(w), B, E, M);
    else
        k_corrector_energy<float><<<(unsigned)P, 256, 0, s>>>(n, h, static_cast<const float *>(w), B, E, M);
    return cudaGetLastError();
}

cudaError_t launch_offdiag_apply(long long P, OffdiagLevel off, const double *B, double *Koff,
                                 cudaStream_t s)
{
    const int th = 128;
    count_launches(1);
    k_offdiag_apply<<<(unsigned)((P + th - 1) / th), th, 0, s>>>(P, off, B, Koff);
    return cudaGetLastError();
}

}  // namespace mlsd
