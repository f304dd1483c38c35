// Internal declarations shared by the translation units of libmlsd.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <algorithm>
#include <vector>

#include "../../include/mlsd.h"

namespace mlsd {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxLevels = 16;

// ---------------------------------------------------------------------------
// Patch solve launch description (one level, all patches).
struct PatchParams {
    const void *band;        // level band grid [Nl][Nl], float or double
    long long Nl;            // band grid points per 2*pi
    int n_macro;
    double h, L;             // patch spacing and side
    const double *Kb;        // [P][3] base diffusivity
    double *S;               // [P][4] time-averaged (S11, S21, S12, S22)
    void *wdump;             // [P][2][n][n] or nullptr
    int *status;             // device status word
    double cfl, t_burn, t_avg;
    long long nb_fixed, na_fixed;
    long long P;             // patches
    long long item0, items;  // work items [item0, item0 + items), item = 2p + (j - 1)
    long long *steps;        // [2P]: n_burn + n_avg, then n_avg, per patch (written by the j = 1 CTA) or nullptr
    const int *pidx;         // patch index of work-item pair (item >> 1), or nullptr: identity
    long long tile = 0;      // 0: band is the level grid; else per-patch tiles, patch p at band + p * tile
    const int *count_dev = nullptr;   // if set: only the first 2 * (*count_dev) items, taken by a
                                      // grid-stride loop (a launch sized before the count is known)
};


// Variant of the patch kernel: thread block shape per patch size and precision.
struct PatchVariant {
    int n, precision, bx, by, minb, packed, threads;   // packed: both fields per CTA (f32x2)
    int cluster;             // CTAs per patch field (slabs of n / cluster rows), 1 = one CTA
    int split;               // split-phase stage barriers (interior cells overlap the barrier)
    int tmem;                // 1: the per-cell coefficients live in tensor memory; 2: the same,
                             // with the column halos read as the rows need them
    size_t smem;
    const void *fn;
};

int patch_variants(int n, int precision, std::vector<PatchVariant> &out);
// the tilings of each patch size, compiled in their own translation units
int patch_variants_n32(int precision, std::vector<PatchVariant> &out);
int patch_variants_n64(int precision, std::vector<PatchVariant> &out);
int patch_variants_cluster(int n, std::vector<PatchVariant> &out);
cudaError_t launch_patch(const PatchVariant &v, const PatchParams &p, long long grid,
                         cudaStream_t s);

// All patches of a level in one persistent launch (patch_level.cu): clusters of
// 4 CTAs of 512 threads with the stencil coefficients in tensor memory take
// tickets of the level's work, each a 256^2 field or four CTA tasks (one 128^2,
// four 64^2 or sixteen 32^2 fields).
struct LevelParams {
    static constexpr int CLUSTER = 4;
    PatchParams cls[4];      // per patch size: 0 = 32, 1 = 64, 2 = 128, 3 = 256 (as present)
    const long long *task;   // [n_tickets][CLUSTER]: (size << 56) | first work item, or -1: none
    long long n_tickets;
};
size_t level_kernel_smem();
cudaError_t level_kernel_clusters(int *out);
cudaError_t launch_level(const LevelParams &lp, int clusters, cudaStream_t s);

// Combine the two fields' flux averages: K = B + sym(S).
cudaError_t launch_compose(long long P, const double *B, const double *S, double *K,
                           int *status, cudaStream_t s);

// ---------------------------------------------------------------------------
// Level chain (Algorithm 3) helpers.
struct OffdiagLevel {
    const double *q12;       // [P][stride] line variances of psi_12 or nullptr
    const double *q21;       // [P][stride] line variances of psi_21 or nullptr
    int stride;              // largest patch size of the level
    const int *np;           // [P] lines (= patch size) per patch, or nullptr: all = stride
};
struct ChainTables {
    int L;
    long long P;
    double kappa;
    OffdiagLevel off[kMaxLevels];
    double *B[kMaxLevels];       // [P][3]  base entering level l from above
    double *Koff[kMaxLevels];    // [P][3]
};
cudaError_t launch_topdown(const ChainTables &t, cudaStream_t s);
// base_l = K_off,l(K*_{l+1} - Koff_l + B_l) (or K_off,L(B_L) at the finest level);
// also writes K*_{l+1} = base_{l+1} + sym(S_{l+1}) when Kstar_next != nullptr.
cudaError_t launch_level_base(long long P, int finest, const double *base_next,
                              const double *S_next, double *Kstar_next, const double *Koff_l,
                              const double *B_l, OffdiagLevel off, double *base_out,
                              cudaStream_t s);
cudaError_t launch_offdiag_apply(long long P, OffdiagLevel off, const double *B, double *Koff,
                                 cudaStream_t s);

// ---------------------------------------------------------------------------
// Band synthesis (set-up): psi on an Nl x Nl lattice from a mode list.
// Modes are grouped by k1: group g holds modes [gofs[g], gofs[g+1]) with
// wavenumber gk1[g]; per mode k2, re, im.
struct ModeGroups {
    int n_groups;
    const int *gk1;          // [n_groups]
    const int *gofs;         // [n_groups + 1]
    const int *k2;           // [n_modes]
    const double *re, *im;   // [n_modes]
};
// G scratch: [n_groups][Nl] double2.  out: float or double [Nl][Nl].
cudaError_t launch_band_synth(const ModeGroups &m, long long Nl, double2 *G, void *out,
                              int out_double, cudaStream_t s);

// Factorised line variances of one off-diagonal part (groups keyed by the
// wavenumber across the line, per-mode k2 field = the one along it);
// Gscratch holds n_macro * groups * n * r double2.
cudaError_t launch_line_var(const ModeGroups &grp, long long Nl, int n, int r, int n_macro,
                            long long count, const int *idx, int along_x2, int stride, double *q,
                            double2 *Gscratch, cudaStream_t s);
// max |v| of a band over every patch's nref x nref reference nodes (v1, v2 on an
// Nr = nref * m lattice)
cudaError_t launch_S_from_K(long long P, const double *base, const double *K, double *S, cudaStream_t s);
cudaError_t launch_corrector_energy(int n, double h, long long P, int precision, const void *w,
                                   const double *B, double *E, double *M, cudaStream_t s);
cudaError_t launch_patch_vmax(const double *v1, const double *v2, long long Nr, int nref,
                              int n_macro, long long P, double *vmax, cudaStream_t s);

// ---------------------------------------------------------------------------
// Periodic component of every patch of a size class (n = 32 or 64, FP32) into
// tiles [P][n][n], indexed by patch (pidx lists the class's patches, or null).
cudaError_t launch_periodize(const float *band, long long Nl, int n, int n_macro, const int *pidx,
                             long long count, float *tiles, cudaStream_t s);

// Failure-path checks of the two bounded device waits (nothing in flight).
cudaError_t launch_wait_check_nbr(int *status, cudaStream_t s);
cudaError_t launch_wait_check_mbar(int *status, cudaStream_t s);
cudaError_t launch_wait_check_tile(int *status, cudaStream_t s);
// tensor-core GEMM D = A B^T of the training step (gemm_tc.cu): mode 0 forward epilogue,
// 1 backward epilogue, 2 partial sums over K slices
cudaError_t gemm_tc(int mode, int M, int N, int K, const void *A, long long lda, const void *B,
                    long long ldb, const float *bias, float *Z, const float *Zprev, void *out,
                    void *outT, int ldT, float *part, int splits, int *slices, int *status,
                    cudaStream_t s);
int gemm_tc_splits(int M, int N, int K, int sms);
// 3-D core-matrix tensor map (CUtensorMap) of a bfloat16 matrix [rows][K], rows ld apart
bool encode_rows_bf16(void *map, const void *base, long long rows, long long K, long long ld,
                      int box_rows);
// 2-D FP32 tensor map (CUtensorMap, 128 bytes) of a row-major [height][width] array
bool encode_f32_2d(void *map, const float *base, long long width, long long height, int box_w,
                   int box_h);
// MLSD_OK, or MLSD_ETIMEOUT when a tile wait of the DNS kernel ran out since the last call
int dns_status_take(cudaStream_t s);
// the DNS kernel the process picked ("" before the first run)
const char *dns_kernel_name();

// ---------------------------------------------------------------------------
// Macro solver and direct simulation.
cudaError_t macro_run(int N, void *U, int precision, const double *K, double dt, int nsteps,
                      double *mass_dev, void *scratch, cudaStream_t s);
cudaError_t macro_run_dirichlet(int N, void *U, int precision, const double *K, double dt,
                                int nsteps, double ul, double ur, double *mass_dev, void *scratch,
                                cudaStream_t s);
cudaError_t dns_run_dirichlet(int nf, void *u, void *u_tmp, const float *psi, int precision,
                              double kappa, double dt, int nsteps, double ul, double ur,
                              cudaStream_t s);
size_t macro_scratch_bytes(int N, int precision, int nsteps);
cudaError_t macro_dt_max(int N, const double *K, double *max_dev, cudaStream_t s);

cudaError_t dns_run(int nf, float *u, float *u_tmp, const float *psi, double kappa, double dt,
                    int nsteps, cudaStream_t s);
cudaError_t dns_vmax(int nf, const float *psi, unsigned *vmax_bits, cudaStream_t s);
cudaError_t coarse_grain(int nf, const float *u, int N, float *U, double *mass_dev,
                         cudaStream_t s);

// Kernel launch counter (host side, all launches of this library).
void count_launches(long long n);
long long launch_count();

// Surrogate (surrogate.cu)
long long sur_param_count(int h);
cudaError_t launch_features(const float *band, long long Nl, long long tile, int n, int n_macro,
                            const int *pidx, long long count, const double *B, double kappa,
                            void *X, float *F32, double *Q, cudaStream_t s);
// ws: split-k partials of the CUDA-core GEMMs, ws_n floats (sur_split_workspace(h) lets
// every training shape split fully; nullptr disables splitting)
long long sur_split_workspace(int h);
cudaError_t sur_forward(int h, int M, const void *X, const float *wf, const void *wb,
                        float *Z[4], void *Aact[3], float *ws, long long ws_n, cudaStream_t s);
cudaError_t sur_grad(int h, int M, const void *X, const float *Y, const float *wf, const void *wb,
                     float *Z[4], void *Aact[3], float *dA, float *dB, float *g, double *part,
                     double *loss_dev, float *ws, long long ws_n, cudaStream_t s);
// buffers of the tensor-core training step (sur_grad_tc); ldT >= max_rows rounded up to 8
struct SurTc {
    int max_rows = 0, ldT = 0;
    __nv_bfloat16 *XT = nullptr;          // [640][ldT]
    __nv_bfloat16 *AT[3] = {};            // [h][ldT] transposed activations
    __nv_bfloat16 *WT[2] = {};            // [h][h] transposed W_1, W_2
    __nv_bfloat16 *dZ[2] = {};            // [max_rows][h] bfloat16 gradients
    __nv_bfloat16 *dZT[2] = {};           // [h][ldT]
};
cudaError_t sur_grad_tc(int h, int M, const void *X, const float *Y, const float *wf,
                        const void *wb, float *Z[4], void *Aact[3], float *dA, float *dB,
                        float *g, double *part, double *loss_dev, float *ws, long long ws_n,
                        const SurTc &tc, int *status, cudaStream_t s);
cudaError_t sur_adam(long long n, float *w, const float *g, float *m, float *v, float lr, int t,
                     void *wb, cudaStream_t s);
cudaError_t sur_to_bf16(long long n, const float *w, void *wb, cudaStream_t s);
// rows idx[r] of (X, Y); with aug, idx[r] = 8 row + g takes the row's image under
// symmetry g of the square (mlsd_surrogate_symmetry)
cudaError_t sur_gather(int M, const int *idx, const void *X, const float *Y, void *Xb, float *Yb,
                       int aug, cudaStream_t s);
cudaError_t sur_symmetry(long long n, int g, const void *X, const float *Y, void *Xo, float *Yo,
                         cudaStream_t s);
cudaError_t sur_add_loss(const double *loss, double *acc, cudaStream_t s);
cudaError_t sur_targets(long long P, const double *B, const double *K, const double *Q, float *Y,
                        cudaStream_t s);
cudaError_t sur_disagree(long long P, int members, const float *out, const double *B,
                         const double *Q, double thr, double *K, int *flag, int *idx, int *count,
                         cudaStream_t s);
cudaError_t sur_merge(int n, const int *idx, const double *B, const double *S, double *K,
                      cudaStream_t s);
cudaError_t sur_merge_dev(long long P, const int *n_dev, const int *idx, const double *B,
                          const double *S, double *K, cudaStream_t s);

// Tensor-core inference (mlp_tc.cu)
size_t mlp_tc_smem();
bool mlp_tc_supported(int h);
cudaError_t launch_mlp_tc(const void *X, long long M, int h, int members, const void *const *wb_dev,
                          const float *const *wf_dev, float *out, int *status, cudaStream_t s);
// TMA-fed variant: weight tensor maps prepared once (host), X map per call
bool mlp_tma_prepare(int h, int members, void *const *wb_host, void *maps_out);
size_t mlp_tma_maps_bytes();
cudaError_t launch_mlp_tma(const void *X, long long M, int h, int members, const void *maps,
                           const float *const *wf_dev, float *out, int *status, cudaStream_t s);

// Shared small device helpers ------------------------------------------------
__host__ __device__ inline long long pmod_ll(long long a, long long m)
{
    long long r = a % m;
    return r < 0 ? r + m : r;
}
// nearest lattice index to i * Nl / N (halves rounded up), minus n/2
__host__ __device__ inline long long patch_origin(long long i, long long N, long long Nl, int n)
{
    return (2 * i * Nl + N) / (2 * N) - n / 2;
}

// psi of patch node (a, b): from the level's band grid at the patch origin
// (periodic wrap), or from the patch's own tile (periodised band, n x n)
template <typename real>
__device__ __forceinline__ real patch_band(const real *band, long long Nl, long long tile,
                                           long long p, long long ox, long long oy, int n, int a,
                                           int b)
{
    return tile ? band[p * tile + (long long)b * n + a]
                : band[pmod_ll(oy + b, Nl) * Nl + pmod_ll(ox + a, Nl)];
}

}  // namespace mlsd
