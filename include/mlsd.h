/*
 * mlsd.h -- C ABI of the GB300 (sm_103a) library for the seamless multiscale
 * estimate of the effective diffusivity of passive advection-diffusion
 *
 *     u_t = v . grad u + kappa Lap u,   div v = 0,   v = (-d psi/dx2, d psi/dx1)
 *
 * (Lee & Engquist, Eq. (model) and Sec. 2.1).  Every call takes plain host or
 * device pointers and sizes; no C++ or framework types cross this boundary.
 *
 * Conventions for every entry point:
 *   - Domain [0, 2*pi)^2, periodic.  Macro grid N x N with nodes X_ij = (iH, jH),
 *     H = 2*pi/N; node (and patch) index p = j*N + i.
 *   - Symmetric tensors are stored as 3 doubles (K11, K12, K22); arrays of them
 *     as [count][3], row-major.
 *   - Fields are row-major [b][a] with a along x1 (fast) and b along x2 (slow).
 *   - Calls are asynchronous on the given CUDA stream (a cudaStream_t passed as
 *     void*, NULL = the legacy default stream) unless stated otherwise.  Device
 *     pointers must stay valid until the stream reaches the call.
 *   - Return 0 on success or a negative MLSD_E* code.  On a host-detected error
 *     (bad argument, allocation failure) nothing is enqueued and output buffers
 *     are left untouched.  Errors found on the device (non-finite result) are
 *     latched in the handle's status word and reported by mlsd_status().
 *   - Output buffers are owned by the caller; the library never frees them.
 *   - A handle is not thread-safe: use one handle per host thread.
 */
#ifndef MLSD_H
#define MLSD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MLSD_OK            0
#define MLSD_EINVAL       -1   /* invalid argument */
#define MLSD_ENOMEM       -2   /* device or host allocation failed */
#define MLSD_ECUDA        -3   /* a CUDA runtime call failed */
#define MLSD_ETIMEOUT     -4   /* a bounded device wait ran out */
#define MLSD_ENONFINITE   -5   /* a NaN or Inf appeared in a result */
#define MLSD_EUNSUPPORTED -6   /* configuration without a compiled kernel */

#define MLSD_FP32 0            /* stencil arithmetic and storage in FP32, averages in FP64 */
#define MLSD_FP64 1            /* everything in FP64 */

#define MLSD_PLAIN     0       /* every patch solved by time stepping */
#define MLSD_SURROGATE 1       /* learned estimate, time stepping as fallback */

/* Problem statement: the stream function, the molecular diffusivity and the
 * level hierarchy (Sec. 3: Fourier decomposition with factor alpha, local
 * domains whose side and grid spacing shrink by the same factor per level).
 *
 *   psi(x) = sum_t Re[(re[t] + i im[t]) exp(i (k1[t] x1 + k2[t] x2))]
 *
 * The mode list must be Hermitian-complete (each mode with its mirror -k and
 * the conjugate coefficient) and must not contain k = 0.  Level l = 1..L
 * (1 = coarsest) owns wavenumber magnitudes in [e_{l-1}, e_l) with the first
 * level's lower bound read as 0 (band_edges = e_0 < e_1 < ... < e_L); a mode
 * whose two magnitudes fall in the same level is part of that level's
 * diagonal band (psi_11 / psi_22), otherwise it is an off-diagonal part
 * (psi_12 or psi_21) of the lower of the two levels.
 * The local domain (patch) of level l is a square of side L_l = 2*pi/m_l
 * centred at the macro node (snapped to the nearest grid node of spacing
 * h_l = L_l/n_l) with an n_l x n_l periodic grid.                           */
typedef struct {
    int n_macro;               /* N >= 1 */
    double kappa;              /* molecular diffusivity, > 0 */
    int n_modes;
    const int32_t *k1, *k2;    /* host arrays [n_modes] */
    const double *re, *im;     /* host arrays [n_modes] */
    int n_levels;              /* L >= 1 */
    const double *band_edges;  /* host [L + 1], increasing */
    const int32_t *patch_div;  /* host [L] integers m_l >= 1, or NULL: m_l = e_{l-1} (must be integer) */
    const int32_t *patch_n;    /* host [L] patch grid sizes: 32, 64, 128 or 256 (FP32); 32 or 64 (FP64) */
    double cfl;                /* micro time-step factor, e.g. 0.2 */
    double t_burn_tau;         /* burn-in length in relaxation times tau, e.g. 8 */
    double t_avg_tau;          /* averaging window in tau, e.g. 4 */
    int64_t n_burn_fixed;      /* if n_avg_fixed > 0: fixed step counts replace the tau rule */
    int64_t n_avg_fixed;
    int precision;             /* MLSD_FP32 or MLSD_FP64 */
    /* Patch sizes per patch (uneven sizes within a level).  A level whose
     * patch_n is 0 takes, per patch, the smallest power of two n in
     * [n_min, n_max] with n >= 10 kmax L / (2 pi) (10 points per wavelength of
     * the level's finest diagonal mode, kmax = max(|k1|, |k2|)) and
     * n >= L vmax / (2 kappa) (cell Peclet number <= 2 with the molecular
     * diffusivity), vmax = max |v| of the level's band over the patch's 32 x 32
     * reference nodes.  patch_n_map, if not NULL, gives every patch's size
     * explicitly ([L][P], overrides patch_n).                                 */
    const int32_t *patch_n_map;
    int n_min, n_max;          /* 0 -> 32, 256 */
    /* Periodisation of the diagonal band on the patches (for a band that is
     * not periodic on its patch, e.g. patches of side 2H, Sec. 3): 0 samples
     * the band and wraps it at the seam; 1 replaces each patch's samples u by
     * their periodic component p of the periodic-plus-smooth decomposition
     * u = p + s (Moisan 2011): the periodic 5-point Laplacian of p equals the
     * Laplacian of u over in-patch neighbours only.  Computed once at set-up
     * into per-patch tiles ([P][n][n] per size class).  FP32, n = 32 or 64;
     * other combinations give MLSD_EUNSUPPORTED.                              */
    int periodize;
} mlsd_problem;

/* Description of one level, as built. */
typedef struct {
    int n;                     /* patch grid n x n */
    int64_t Nl;                /* grid points per 2*pi at this level: h = 2*pi/Nl, L = n h */
    double L, h;
    int64_t n_patches;         /* = N*N */
    int n_diag_modes, n_off12_modes, n_off21_modes;
    int tile_bx, tile_by;      /* cells per thread of the patch kernel the autotuner chose */
    int threads;               /* threads per CTA of that kernel */
    int packed;                /* 1: one CTA per patch, both fields in f32x2 pairs; 0: one per field */
    int cluster;               /* CTAs (a thread-block cluster) sharing one patch field, in row slabs */
    int min_ctas;              /* register cap of the kernel: at least this many CTAs per SM */
    int split;                 /* stage synchronisation: 0 one barrier per stage (cluster-wide
                                  when cluster > 1); 1 split-phase barriers (interior cells
                                  computed while the barrier completes); 2 neighbour signalling
                                  (cluster > 1: a CTA barrier, and mbarrier arrivals from the two
                                  neighbouring slabs for the halo rows they push); 3 bulk row
                                  copies (cluster > 1: a CTA barrier, and the two halo rows moved
                                  by cp.async.bulk completing on the receiver's mbarrier); 4 the
                                  row-paired f32x2 kernel (not a synchronisation mode: one
                                  barrier per stage, two cells per FFMA2); 5 bulk row copies
                                  with the rows that need a neighbour's row computed last, so
                                  that the copies land while the others are computed */
    int n_classes;             /* patch sizes in the level; n, Nl, h and the tile fields describe
                                  the class with the most work; all classes run concurrently */
    int coef_tmem;             /* 1: the kernel keeps the two per-cell stencil coefficients in
                                  the SM's tensor memory instead of registers (two registers per
                                  cell instead of four, so a field needs half the SMs); 2: the
                                  same, with the halo columns read as the rows need them */
    int level_launch;          /* 0: one launch per patch size; 1, 2: every patch of the level in
                                  one persistent launch (clusters of 4 CTAs of 512 threads with the
                                  coefficients in tensor memory take tickets of 65 536 cells: a
                                  256^2 field, or per CTA one 128^2, four 64^2 or sixteen 32^2
                                  fields), 256^2 tickets first (1) or spread among the others (2) */
} mlsd_level_desc;

typedef struct mlsd_levels mlsd_levels;   /* opaque; owns all device tables and scratch */

/* Validate the problem, decompose the spectrum (Sec. 3.1), synthesise every
 * level's diagonal band on the device, and precompute the line variances that
 * Algorithm 1 needs.  Allocates device memory; blocks until set-up is done.
 * Set-up also picks the thread-block tiling of the patch kernel per patch
 * size: every compiled candidate is timed on a sample of the level's patches
 * (a short fixed window) and the fastest is kept for the process; the
 * environment variable MLSD_TILE=<bx>x<by>[m<min CTAs/SM>][c<cluster>][p][s|n|b|d|r][t|l]
 * forces one where it exists for the level's patch size (p: the packed kernel
 * that advances both fields of a patch in f32x2 pairs; c: CTAs per patch field;
 * s: split-phase stage barriers; n: neighbour signalling between the slabs of
 * a cluster instead of a cluster-wide barrier; b: the slab edge rows moved by
 * bulk copies that complete on the receiver's mbarrier; d: as b, with the rows
 * that need a neighbouring slab's row computed after the others; r: rows r and r + by/2
 * of a thread's block in f32x2 pairs, one FFMA2/FADD2 per two cells; t: the two per-cell
 * coefficients of the stencil held in tensor memory, loaded a block row at a
 * time, instead of registers; l: as t, with the west and east halo columns read
 * two rows at a time as the row loop reaches them).  MLSD_TUNE_LOG set to
 * anything prints every candidate's trial time to stderr.
 * Patch sizes 32 and 64 run one CTA per field (or per patch, packed); 128 and
 * 256 split each field over a thread-block cluster of 2-16 CTAs that exchange
 * their slab edges through distributed shared memory, or, with the
 * coefficients in tensor memory, run a 128 field in one CTA of 512 threads.
 * An FP32 level with several patch sizes (all among 32, 64, 128, 256) is also
 * timed as one persistent launch of every patch, with two patch-to-cluster
 * orders, against the per-size launches, and the fastest is kept
 * (MLSD_LEVEL = 0 keeps the per-size launches, 1 or 2 forces the one launch
 * with 256^2 fields first or interleaved; mlsd_level_desc.level_launch).
 * Returns MLSD_EINVAL for an invalid problem, MLSD_EUNSUPPORTED for a patch
 * size or precision without a kernel, MLSD_ENOMEM / MLSD_ECUDA otherwise.   */
int mlsd_build_levels(const mlsd_problem *p, void *cuda_stream, mlsd_levels **out);

/* Free a handle (synchronises with its work first).  NULL is ignored. */
void mlsd_free_levels(mlsd_levels *h);

int mlsd_level_info(const mlsd_levels *h, int level, mlsd_level_desc *out);

/* Patch size of every patch of a level: n_out_host [P].  Host only.       */
int mlsd_patch_sizes(const mlsd_levels *h, int level, int32_t *n_out_host);

/* One level of patch solves: the numerical homogenization K[psi_l, B; Omega_l]
 * of Sec. 2.2 for every macro node at once.  For each patch and each
 * gradient G = e_j (j = 1, 2) the fluctuation w_j (u = G.x + w_j, w_j periodic
 * on the patch, w_j(0) = 0) is advanced with Heun's RK2 on the second-order
 * central-difference operator
 *     w_t = v.(grad_h w + G) + B11 Dxx w + 2 B12 Dxy w + B22 Dyy w
 * for n_burn + n_avg steps; the spatial mean of v_i w_j after each of the last
 * n_avg steps is averaged in FP64 into S_ij and
 *     K11 = B11 + S11,  K22 = B22 + S22,  K12 = B12 + (S12 + S21)/2.
 * The time step is cfl * min(h / max(|v1|+|v2|), h^2 / (2 tr B + 4|B12|)),
 * capped by the RK2 stability bound (8 lambda_min h^2 / vmax^4)^(1/3); the
 * window is t_burn_tau and t_avg_tau relaxation times L^2/(4 pi^2 lambda_min(B))
 * (or the fixed step counts of the problem).
 *   level      1..L
 *   K_base_dev device [P][3] base diffusivity B per patch (symmetric positive definite)
 *   K_out_dev  device [P][3] result; may not alias K_base_dev
 *   w_dump_dev device [P][2][n][n] of float (MLSD_FP32) or double (MLSD_FP64)
 *              receiving the final w_1, w_2 of every patch, or NULL; only for
 *              a level with one patch size (else MLSD_EINVAL)                */
int mlsd_solve_level(mlsd_levels *h, int level, const double *K_base_dev, double *K_out_dev,
                     void *w_dump_dev, void *cuda_stream);

/* Energy diagnostic of a level's correctors (HMM step 3, the energy form of
 * the estimator): from the w_dump of an mlsd_solve_level call with the same
 * base, per patch
 *   E_jk = < B11 D+x w_j D+x w_k + B12 (D0x w_j D0y w_k + D0y w_j D0x w_k)
 *            + B22 D+y w_j D+y w_k >,
 * with D+ forward and D0 central differences (periodic on the patch), and the
 * means <w_j>.  Multiplying the steady corrector equation by w_k and summing by
 * parts gives E = K - B at steady state up to the O(h^2) part of the central
 * advection term, which is not skew-adjoint on the grid (exactly for shear
 * flows, whose correctors are not advected): E against the flux estimate is a
 * resolution and relaxation check.  Evaluated on the final corrector, not
 * summed over the window.
 *   K_base_dev device [P][3]; w_dump_dev device [P][2][n][n] (float for MLSD_FP32,
 *   double for MLSD_FP64); E_out_dev device [P][3] (E11, E12, E22);
 *   mass_out_dev device [P][2] or NULL.  One patch size per level (else
 *   MLSD_EINVAL).                                                           */
int mlsd_corrector_energy(mlsd_levels *h, int level, const double *K_base_dev,
                          const void *w_dump_dev, double *E_out_dev, double *mass_out_dev,
                          void *cuda_stream);

/* Algorithms 1-2 of level l for every patch: each off-diagonal part is treated
 * as a shear on every patch line (Eq. shearhomoX/Y with base B), the line
 * values are combined by the layered-medium harmonic mean, and
 *     K_off = K[psi_12; B] + K[psi_21; B] - B.
 * Identity where the level has no off-diagonal part.
 *   B_dev, Koff_dev  device [P][3]; may alias.                              */
int mlsd_offdiag(mlsd_levels *h, int level, const double *B_dev, double *Koff_dev,
                 void *cuda_stream);

/* Algorithm 3 over the whole hierarchy, finest level first, for every macro node:
 *   B_1 = kappa I, Koff_l = K_off,l(B_l), B_{l+1} = Koff_l;
 *   K*_L = K[psi_L; K_off,L(B_L)];
 *   K*_l = K[psi_l; K_off,l(K*_{l+1} - Koff_l + B_l)] for l = L-1 .. 1;
 *   K_macro = K*_1.
 *   mode            MLSD_PLAIN, or MLSD_SURROGATE: the levels with an attached
 *                   surrogate (mlsd_attach_surrogate) take mlsd_solve_level_surrogate's
 *                   K* (ensemble, plain solves where the members disagree), the
 *                   others the plain solve; MLSD_EINVAL if no level has one.
 *                   This mode blocks once per surrogate level and is not captured
 *                   in a graph.
 *   K_macro_dev     device [P][3]
 *   K_levels_dev    device [L][P][3] receiving K*_l, or NULL
 * The first call (and any call with other output pointers) captures the
 * whole sequence -- every level's kernels, with concurrent size classes on
 * forked streams -- into a CUDA graph on an internal stream; later calls
 * replay it on cuda_stream.  With profiling on (mlsd_profile) or the
 * environment variable MLSD_NO_GRAPH set, the kernels are launched directly. */
int mlsd_effective_diffusivity(mlsd_levels *h, int mode, double *K_macro_dev,
                               double *K_levels_dev, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Learned surrogate of the patch solve (not in the paper).  A small ensemble
 * of MLPs maps a patch's features to the part of K that the resummed
 * perturbation series E below misses; where the members disagree, or the
 * series is far from converged, the plain patch solve above is run instead.
 *
 * Perturbation moments.  At steady state the corrector of field j solves
 * (L0 + A) w_j = -v_j, L0 = B11 D+D-x + 2 B12 D0x D0y + B22 D+D-y (Fourier
 * symbol -D(k)/h^2, D = B11 (2 - 2 cos t1) + B22 (2 - 2 cos t2) + 2 B12 s1 s2,
 * t_i = 2 pi k_i / n, s_i = sin t_i), A w = v1 D0x w + v2 D0y w.  Expanding in
 * v: c_j^0 = -L0^{-1} v_j, c_j^m = -L0^{-1} A c_j^{m-1}, and K - B = sum of
 *   T_m = sym <v_i c_j^{m-2}>  (m >= 2; T_2 is the small-Peclet limit).
 * The library computes T_2..T_19 on the feature grid with FFTs and resums
 * the series where it diverges: with the pairs
 * p_k = T_(2k+2) + T_(2k+3), the [K/K] Pade approximant at 1 of sum_k p_k x^k
 * (Wynn's epsilon algorithm on the partial sums) for K = 2, 3, 4; the
 * estimate is E = [4/4], and gap = max_c |[4/4]_c - [3/3]_c| measures how far
 * it is from converged.
 *
 * Feature grid: the patch nodes for n = 32 and 64; for n = 128 and 256 the
 * nf = 64 x 64 sub-lattice of every (n/64)-th node (psi and the moments are
 * taken there; a band resolved on the patch is resolved on the sub-lattice:
 * its modes up to the window's 8 are exact, and the moments converge like
 * the grid).
 * Features of a patch (MLSD_SUR_FEATURES = 606 values, stored as one bfloat16
 * row of MLSD_SUR_IN = 640, zero padded):
 *   [0, 578)  Re and Im of the DFT on the feature grid (nf nodes a side)
 *               psihat(k) = nf^-2 sum_ab (psi[b][a] - mean psi) exp(-2 pi i (k1 a + k2 b)/nf)
 *             of the level's band, k2 = -8..8 (slow),
 *             k1 = -8..8, each times MLSD_SUR_PSI_SCALE / (tr(B)/2);
 *   578..580  B11/kappa, B12/kappa, B22/kappa;   581  log kappa;
 *   582..596  asinh(MLSD_SUR_T_SCALE T_m / tr(B)), m = 2..6, components 11, 12, 22;
 *   597..605  asinh(MLSD_SUR_T_SCALE x / tr(B)) for x = [2/2], [3/3], [4/4].
 * Network output (the training target):
 *   asinh((K - B - E) MLSD_SUR_Y_SCALE / tr(B)).
 * Member network: 640 -> h -> h -> h -> 3, exact-erf GELU after the first three
 * layers, bfloat16 weights and activations, FP32 accumulation.  Parameters of
 * a member in one FP32 array, row-major (out x in):
 *   W1[h][640] b1[h] W2[h][h] b2[h] W3[h][h] b3[h] W4[3][h] b4[3].         */
#define MLSD_SUR_IN 640
#define MLSD_SUR_FEATURES 606
#define MLSD_SUR_PSI_SCALE 32.0
#define MLSD_SUR_T_SCALE 10.0
#define MLSD_SUR_Y_SCALE 300.0
#define MLSD_SUR_GAP_WEIGHT 0.3
typedef struct mlsd_surrogate mlsd_surrogate;

int64_t mlsd_surrogate_param_count(int hidden);          /* per member */
/* members >= 1, hidden a multiple of 32 (<= 512), max_batch rows per call of
 * the training kernels (prediction is chunked by it).  Weights start at 0.  */
int mlsd_surrogate_create(int members, int hidden, int max_batch, mlsd_surrogate **out);
void mlsd_surrogate_free(mlsd_surrogate *s);
/* host FP32 parameter arrays (layout above); set resets the Adam state      */
int mlsd_surrogate_set_params(mlsd_surrogate *s, int member, const float *params_host);
int mlsd_surrogate_get_params(mlsd_surrogate *s, int member, float *params_host);
/* Features of every patch of a level (one patch size per level, n = 32, 64,
 * 128 or 256; FP32) with base B_dev [P][3]: X_dev bfloat16 [P][640]; F32_dev
 * [P][606] or NULL.  Levels of several sizes: MLSD_EUNSUPPORTED.            */
int mlsd_surrogate_features(mlsd_levels *h, int level, const double *B_dev, void *X_dev,
                            float *F32_dev, void *cuda_stream);
/* Mean-squared-error loss of one member on M <= max_batch rows (X bfloat16
 * [M][640], Y [M][3]) and its gradient grad_dev (FP32, parameter layout; NULL
 * to skip).  Blocks for the loss.                                          */
int mlsd_surrogate_grad(mlsd_surrogate *s, int member, const void *X_dev, const float *Y_dev,
                        int M, float *grad_dev, double *loss_host, void *cuda_stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected) of one member on
 * a batch; loss_host (or NULL) receives the batch loss before the step.     */
int mlsd_surrogate_train_step(mlsd_surrogate *s, int member, const void *X_dev,
                              const float *Y_dev, int M, float lr, double *loss_host,
                              void *cuda_stream);
/* Training data of one level, all on the device: the plain patch solve of
 * every patch with base B_dev [P][3], its features X_dev (bfloat16 [P][640])
 * and targets Y_dev (FP32 [P][3]) = asinh((K - B - E) MLSD_SUR_Y_SCALE / tr(B)),
 * E the resummed series estimate in FP64.  Same level limits as
 * mlsd_surrogate_features.                                                  */
int mlsd_surrogate_dataset(mlsd_levels *h, int level, const double *B_dev, void *X_dev,
                           float *Y_dev, void *cuda_stream);
/* The symmetry group of the square acting on training rows: element g (0..7)
 * reflects x1 (bit 0: grid index a -> -a mod n), then x2 (bit 1), then swaps
 * x1 and x2 (bit 2).  The patch problem is equivariant under it: psi maps to
 * -psi on the mapped grid for a reflection or a swap (a stream function is a
 * pseudo-scalar), v = (-psi_x2, psi_x1) maps as a vector, the central
 * differences, the periodic wrap, dt and the windows are unchanged, and every
 * symmetric tensor (B, T_m, the approximants, K, the target) maps as R T R^T
 * (asinh is odd, so the stored features and targets map the same way).  So the image of a
 * plain-solved row is the exact row of the mapped patch.  On a row: DFT entry
 * (k1, k2) takes sign * entry (k1s, k2s), (q1, q2) = bit 2 ? (k2, k1) : (k1, k2),
 * k1s = bit 0 ? -q1 : q1, k2s = bit 1 ? -q2 : q2, sign = (-1)^(bits set);
 * tensors (T11, T12, T22) -> (T11, s T12, T22), s = (-1)^(bit 0 + bit 1), then
 * T11 <-> T22 if bit 2; log kappa and the padding are unchanged.
 * mlsd_surrogate_symmetry writes the images under g of n_rows rows (X_out
 * bfloat16 [n][640], Y_out FP32 [n][3]; either output may be NULL with its
 * input); the outputs must not overlap the inputs.                         */
int mlsd_surrogate_symmetry(const void *X_dev, const float *Y_dev, int64_t n_rows, int g,
                            void *X_out, float *Y_out, void *cuda_stream);
/* Train every member with Adam on the n_rows rows of (X_dev, Y_dev) for
 * `epochs` passes in batches of `batch` (<= max_batch) rows.  With augment != 0
 * every row also enters through its 7 other images under the symmetry group
 * above (8 n_rows rows per epoch, mapped as they are gathered; n_rows <=
 * 2^28 - 1), else n_rows rows per epoch; rows / batch steps per epoch.  Each
 * member draws its own row order per epoch (Fisher-Yates on a SplitMix64
 * stream seeded from `seed` and the member index; the rows are gathered on
 * the device); the learning rate decays geometrically from lr to lr_final over
 * the run.  losses_host (or NULL) receives each member's mean batch loss over
 * the last epoch.  Blocks at the end of each member.
 * Arithmetic of a step (and of mlsd_surrogate_grad / _train_step): bfloat16
 * inputs, weights and hidden activations, FP32 accumulation, the hidden
 * layers' pre-activation gradients dZ rounded to bfloat16.  The hidden layers'
 * contractions run on the tensor cores (tcgen05, operands by tensor copies)
 * where the handle could encode tensor maps at creation; MLSD_TRAIN_CUDA set
 * at creation keeps every GEMM on the CUDA cores.                           */
int mlsd_surrogate_train(mlsd_surrogate *s, const void *X_dev, const float *Y_dev, int64_t n_rows,
                         int epochs, int batch, float lr, float lr_final, uint64_t seed,
                         int augment, double *losses_host, void *cuda_stream);
/* Checkpoint: every member's FP32 parameters in one file (magic "MLSDSUR1",
 * int64 members, hidden, parameter count, then the arrays).  load requires
 * the same members and width and resets the Adam state; MLSD_EINVAL on any
 * file or shape mismatch.  Both synchronise the device.                     */
int mlsd_surrogate_save(mlsd_surrogate *s, const char *path);
int mlsd_surrogate_load(mlsd_surrogate *s, const char *path);
/* Inference engine: MLSD_SUR_TENSOR (default where the width allows: one
 * tcgen05 kernel running all layers of a member on 128-row tiles, bfloat16
 * operands in shared memory, FP32 accumulators in tensor memory) or
 * MLSD_SUR_CUDA (the FP32-FMA kernels the training uses).                   */
#define MLSD_SUR_CUDA 0
#define MLSD_SUR_TENSOR 1
int mlsd_surrogate_set_engine(mlsd_surrogate *s, int engine);
/* Device errors of the tensor-core engine (a bounded wait that ran out:
 * MLSD_ETIMEOUT); synchronises, returns and clears the first one.          */
int mlsd_surrogate_status(mlsd_surrogate *s, void *cuda_stream);
/* Every member on M rows: out_dev FP32 [members][M][3].                     */
int mlsd_surrogate_predict(mlsd_surrogate *s, const void *X_dev, int64_t M, float *out_dev,
                           void *cuda_stream);
/* One level with the surrogate: features (with E), ensemble,
 *     K_m = B + E + tr(B) sinh(out_m) / MLSD_SUR_Y_SCALE;
 * a patch whose members disagree or whose resummation has not converged,
 *     max(max_{m,c} |K_m,c - mean_m K_m,c|, MLSD_SUR_GAP_WEIGHT gap)
 *         > threshold * ||mean K||_F,
 * is solved by the plain patch solve (mlsd_solve_level's kernel) instead; the
 * rest take the ensemble mean.  n_fallback_out receives the number of plain
 * solves.  Blocks once (to size the fallback launch).                       */
int mlsd_solve_level_surrogate(mlsd_levels *h, mlsd_surrogate *s, int level,
                               const double *K_base_dev, double *K_out_dev, double threshold,
                               int64_t *n_fallback_out, void *cuda_stream);

/* Attach a trained surrogate to a level for MLSD_SURROGATE chains, with its
 * disagreement threshold (as in mlsd_solve_level_surrogate); s = NULL detaches.
 * The handle keeps the pointer, not the surrogate: the caller keeps it alive
 * while attached.  Same level limits as mlsd_surrogate_features
 * (MLSD_EUNSUPPORTED otherwise).                                            */
int mlsd_attach_surrogate(mlsd_levels *h, int level, mlsd_surrogate *s, double threshold);
/* Plain fallback solves of a level in the last MLSD_SURROGATE chain (-1 if
 * none ran since the surrogate was attached).                               */
int mlsd_surrogate_fallbacks(mlsd_levels *h, int level, int64_t *n_out);

/* Synchronise the handle's stream and return the first error latched on the
 * device since the last call (MLSD_ENONFINITE ...), then clear it.          */
int mlsd_status(mlsd_levels *h, void *cuda_stream);

/* Failure-path check of the library's bounded device waits (failure
 * detection; the paper has no counterpart).  Launches one CTA on the stream
 * that waits on an mbarrier which never receives an arrival, with nothing
 * else in flight:
 *   which = 0: the wait of the cluster-split patch kernels' slab exchanges;
 *   which = 1: the wait of the tensor-core inference kernels;
 *   which = 2: the tile wait of the persistent DNS kernels.
 * Each wait gives up after about a second of SM clocks and latches
 * MLSD_ETIMEOUT in the handle's status word, exactly as on a real failure;
 * mlsd_status then reports it (and clears it), and the context stays usable.
 * Returns MLSD_OK once launched; MLSD_EINVAL for another `which`.           */
int mlsd_check_wait_timeout(mlsd_levels *h, int which, void *cuda_stream);

/* Macro solver for Eq. (homo), U_t = div(K grad U), HMM step 4: conservative
 * flux form on the periodic N x N grid with face tensors
 * K_f = (K_node + K_neighbour)/2 (full tensor, 9-point), Heun's RK2.
 *   U_dev       device [N][N], float (MLSD_FP32) or double (MLSD_FP64), in place
 *   K_dev       device [N*N][3]
 *   dt, nsteps  time step and number of steps (nsteps >= 0)
 *   mass_out    host [nsteps + 1] or NULL: H^2 * sum(U) after each step (FP64);
 *               when non-NULL the call blocks until the steps are done.
 * Allocates (stream-ordered) a device scratch of N*N reals plus the mass list. */
int mlsd_macro_step(int n_macro, void *U_dev, int precision, const double *K_dev, double dt,
                    int nsteps, double *mass_out_host, void *cuda_stream);

/* The macro step with the boundary conditions of the paper's numerical
 * examples (Sec. 4): Dirichlet in x1, periodic in x2.  The paper's [0,1]^2 is
 * posed here as [0, 2 pi] x [0, 2 pi) (x -> 2 pi x, t -> 4 pi^2 t, psi
 * unchanged, kappa unchanged).  Nodes x1 = i H, H = 2 pi / N:
 *   column i = 0 of U is the boundary x1 = 0: set to u_left on entry and held;
 *   the boundary x1 = 2 pi is a virtual column N with the value u_right;
 *   columns 1..N-1 follow the interior scheme of mlsd_macro_step unchanged.
 * K_dev is a periodic field (the level chain's output), so the face tensor
 * between column N-1 and the boundary is (K(N-1) + K(0)) / 2.  Other
 * arguments, the mass list (H^2 sum(U), not conserved here) and the errors
 * are those of mlsd_macro_step.                                             */
int mlsd_macro_step_dirichlet(int n_macro, void *U_dev, int precision, const double *K_dev,
                              double dt, int nsteps, double u_left, double u_right,
                              double *mass_out_host, void *cuda_stream);

/* Stable macro time step dt = cfl H^2 / max_nodes(K11 + K22 + |K12|).
 * Blocks until it is known.                                                 */
int mlsd_macro_dt(int n_macro, const double *K_dev, double cfl, double *dt_out_host,
                  void *cuda_stream);

/* Stream function of a mode list on the full nf x nf grid (nodes 2*pi*a/nf):
 * psi_dev device [nf][nf] float.  Blocks until done (device staging).       */
int mlsd_grid_psi(int n_modes, const int32_t *k1, const int32_t *k2, const double *re,
                  const double *im, int nf, float *psi_dev, void *cuda_stream);

/* Direct simulation of Eq. (model) on the full nf x nf grid (the Sec. 4
 * reference: second-order central differences, second-order Runge-Kutta):
 * u_t = v.grad_h u + kappa Lap_h u with v from psi by central differences,
 * Heun's RK2, nsteps steps.  u_dev [nf][nf] float in place; u_tmp_dev is a
 * caller-provided work field of the same size.  nf a multiple of 128.
 * One fused launch per step; the kernel (per-tile CTAs staged by cp.async, or
 * persistent CTAs fed by tensor copies) is picked once per process by timing
 * each on the caller's grid (MLSD_DNS_TY = 64 | 32 | t32 | t32x2 | t64 | t32p pins
 * one).  The persistent kernels take tiles from a per-device queue: one DNS
 * run at a time per device.  Asynchronous: a tile copy that never lands (a
 * wait of about a second runs out) is reported by mlsd_dns_status.           */
int mlsd_dns_run(int nf, float *u_dev, float *u_tmp_dev, const float *psi_dev, double kappa,
                 double dt, int nsteps, void *cuda_stream);

/* Synchronise the stream and return MLSD_ETIMEOUT if a tile wait of a DNS
 * kernel ran out since the last call (u is then undefined), else MLSD_OK;
 * clears the flag.  MLSD_ECUDA if the stream reports an error.               */
int mlsd_dns_status(void *cuda_stream);

/* Name of the DNS kernel this process picked for mlsd_dns_run ("" before the
 * first run), e.g. "k_dns_tma<32,1>": static storage, not to be freed.      */
const char *mlsd_dns_kernel(void);

/* The direct simulation with the Sec. 4 boundary conditions (Dirichlet in x1,
 * periodic in x2), posed on [0, 2 pi] x [0, 2 pi) as mlsd_macro_step_dirichlet:
 * column 0 of u_dev is set to u_left and held, the virtual column nf has the
 * value u_right; psi (and so v) stays periodic.  One launch per RK stage (the
 * paper's 512 x 512 reference, L2-resident); any nf >= 4.
 *   u_dev, u_tmp_dev  device [nf][nf], float (MLSD_FP32) or double (MLSD_FP64);
 *                     u_tmp_dev is a caller-provided work field
 *   psi_dev           device [nf][nf] float (mlsd_grid_psi)
 * FP64 exists for the paper's long runs (~5e5 steps at its time step): there
 * the FP32 increments of a nearly relaxed profile fall below half an ulp and
 * the field stops diffusing.  Asynchronous on the stream.                   */
int mlsd_dns_run_dirichlet(int nf, void *u_dev, void *u_tmp_dev, const float *psi_dev,
                           int precision, double kappa, double dt, int nsteps, double u_left,
                           double u_right, void *cuda_stream);

/* Stable DNS time step: dt = cfl * min(h / max(|v1| + |v2|), h^2 / (4 kappa)),
 * v from psi by central differences, h = 2*pi/nf.  Blocks until known.    */
int mlsd_dns_dt(int nf, const float *psi_dev, double kappa, double cfl, double *dt_out_host,
                void *cuda_stream);

/* Box average of the fine field onto the macro grid: node (i, j) averages the
 * r x r fine nodes i*r - r/2 .. i*r + r/2 - 1 (periodic), r = nf/N.
 *   U_dev device [N][N] float; mass_out_host (or NULL): h^2 * sum(u) in FP64
 *   (blocks when non-NULL).                                                 */
int mlsd_coarse_grain(int nf, const float *u_dev, int n_macro, float *U_dev,
                      double *mass_out_host, void *cuda_stream);

/* Coarse-graining that allocates nothing (no counterpart in the paper).
 * Same inputs, outputs and results as mlsd_coarse_grain, for callers that
 * cannot call cudaMalloc or a stream-ordered allocator (code running where
 * allocation is forbidden or would break their own memory accounting).  The
 * FP64 box sums and the mass use a fixed scratch array in the library's device
 * memory, 1 + MLSD_NOALLOC_MAX_MACRO^2 doubles (~512 KiB) held on every device
 * that loads the library until the process exits.
 *   n_macro > MLSD_NOALLOC_MAX_MACRO -> MLSD_EINVAL, nothing enqueued.
 * The first call on a device looks up the scratch address there (a host-side
 * query, no allocation); make that first call before any stream capture.
 * All calls share the one scratch array: calls whose work overlaps on the
 * GPU (different streams, or different host threads) race and may corrupt
 * each other's mass and box sums.  Every call overwrites all of the scratch it
 * uses, so no state carries over between calls.  Blocks when mass_out_host is
 * non-NULL.                                                                 */
#define MLSD_NOALLOC_MAX_MACRO 256
int mlsd_coarse_grain_noalloc(int nf, const float *u_dev, int n_macro, float *U_dev,
                              double *mass_out_host, void *cuda_stream);

/* Work done by the last solve of a level (mlsd_solve_level or the level's part
 * of mlsd_effective_diffusivity): cell_updates = sum over patches and the two
 * fields of n^2 (n_burn + n_avg) (one cell of one field advanced one full RK2
 * step), the part of it inside the averaging window (sum of n^2 n_avg over
 * patches and fields: the updates that also add to the flux sums), and the
 * largest per-patch step count.  Any out pointer may be NULL.  Synchronises
 * the stream.                                                               */
int mlsd_level_work(mlsd_levels *h, int level, int64_t *cell_updates_out,
                    int64_t *window_updates_out, int64_t *max_steps_out,
                    void *cuda_stream);

/* The ticket list of the one-launch level kernel (mlsd_level_desc.level_launch)
 * for a level with n_classes patch sizes patch_n[i] (32, 64, 128 or 256, each
 * once) holding patches[i] patches: 4 codes per ticket, one per CTA of a
 * cluster, each (size << 56) | first work item or -1, size 0..3 for 32 .. 256
 * and work item 2q + j - 1 for field j of the class's q-th patch.  A 256^2
 * field is one ticket (the same code 4 times); the other sizes form CTA tasks
 * of 65 536 cells (one 128^2, four 64^2 or sixteen 32^2 fields from the given
 * item on), four per ticket, larger sizes first.  schedule 0 puts every 256^2
 * ticket first, 1 spreads them evenly among the others.  Host only: writes
 * *n_tickets_out always and codes_out [capacity] (4 per ticket) when it fits;
 * MLSD_EINVAL for invalid arguments or too small a capacity.                */
int mlsd_level_schedule(const int32_t *patch_n, const int64_t *patches, int n_classes, int schedule,
                        int64_t capacity, int64_t *codes_out, int64_t *n_tickets_out);

/* Kernel timing of the patch solves: when enabled, every patch-solve launch of
 * the handle is bracketed by CUDA events recorded on the launching stream.
 * enable = 2 also runs the size classes of a level one after another on the
 * caller's stream instead of concurrently, so that each class's events time it
 * alone (per-class rates; the level then takes longer than without profiling).
 * mlsd_profile_collect synchronises, returns the summed device time (ms) and
 * the number of patch-solve launches of the level since the last collect, and
 * clears them.  mlsd_profile_collect_classes does the same per patch size:
 * patch_n_out, kernel_ms_out, launches_out [capacity] receive, for each patch
 * size launched, the size (0 for a launch of every class at once, see
 * mlsd_level_desc.level_launch), its summed device time and its launches;
 * *n_written the number of sizes.  MLSD_EINVAL (nothing cleared) when capacity
 * is too small.  Host arrays, caller-owned.                                 */
int mlsd_profile(mlsd_levels *h, int enable);
int mlsd_profile_collect(mlsd_levels *h, int level, double *kernel_ms_out,
                         int64_t *launches_out);
int mlsd_profile_collect_classes(mlsd_levels *h, int level, int capacity, int32_t *patch_n_out,
                                 double *kernel_ms_out, int64_t *launches_out,
                                 int32_t *n_written);

/* Number of CUDA kernels this library has launched since it was loaded
 * (process-wide counter, host side).                                        */
int64_t mlsd_launch_count(void);

const char *mlsd_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* MLSD_H */
