/*
 * mlsd_oracle.c -- plain, slow FP64 CPU oracle of the seamless multiscale
 * method for passive advection-diffusion (Lee & Engquist).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant generator
 * with the CUDA library.
 *
 * Conventions (the library's, restated here independently):
 *   domain [0, 2*pi)^2, periodic; fields are stored row-major [b][a] with a
 *   along x1 (fast) and b along x2 (slow).
 *   psi(x) = sum_modes Re[(re + i im) exp(i k.x)] over a Hermitian mode list.
 *
 * Every routine below follows one step of the paper:
 *   orc_band_of         -- Fourier decomposition, Sec. 3.1 (psi_11, psi_12,
 *                          psi_21, psi_2, repeated with alpha^2, alpha^3 ...)
 *   orc_patch_psi       -- local domains of the level hierarchy, Sec. 3
 *   orc_velocity        -- v = (-d psi/dx2, d psi/dx1), Sec. 2.1
 *   orc_patch_k         -- numerical homogenization K[psi, B; D]: two linear
 *                          reconstructions with orthogonal gradients, periodic
 *                          fluctuation, evolution to quasi-stationarity, flux
 *                          averaging (HMM steps 1-3, Sec. 2.2)
 *   orc_offdiag_q / orc_offdiag_apply
 *                       -- Algorithm 1 (shear closed form per line, harmonic
 *                          mean across lines) and Algorithm 2 (sum of the two
 *                          off-diagonal effects minus the common base)
 *   orc_chain           -- Algorithm 3 applied level by level, finest first
 *   orc_macro_run       -- macro solver for U_t = div(K grad U), Eq. (homo)
 *   orc_dns_run         -- direct simulation of Eq. (model) on the full grid
 *   orc_macro_run_dirichlet / orc_dns_run_dirichlet
 *                       -- the same two solvers with the Sec. 4 boundary
 *                          conditions (Dirichlet in x1, periodic in x2)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

void orc_periodic_smooth(int n, const double *u, double *p);

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: Fourier decomposition.                                          */
/*                                                                           */
/* Level l (1-based) owns wavenumber magnitudes in [lo_l, e_l) where          */
/* lo_1 = 0 and lo_l = e_{l-1} (the paper's "<= alpha" read with             */
/* lower-inclusive integer edges).  For a mode with la = level(|k1|) and     */
/* lb = level(|k2|):                                                         */
/*   la == lb  -> diagonal part of level la            (psi_11 at that level)*/
/*   la <  lb  -> off-diagonal psi_12 of level la (|k1| low, |k2| high)      */
/*   la >  lb  -> off-diagonal psi_21 of level lb (|k1| high, |k2| low)      */
/* A magnitude at or above the last edge counts as "above every level".      */
/* kind: 0 diagonal, 1 psi_12, 2 psi_21, -1 dropped (both parts too fine).   */
/* ------------------------------------------------------------------------ */
static int level_of_mag(int m, int n_levels, const double *edges)
{
    for (int l = 1; l <= n_levels; ++l) {
        double lo = (l == 1) ? 0.0 : edges[l - 1];
        if ((double)m >= lo && (double)m < edges[l]) return l;
    }
    return n_levels + 1;
}

void orc_band_of(int n_modes, const int *k1, const int *k2, int n_levels,
                 const double *edges, int *level, int *kind)
{
    for (int t = 0; t < n_modes; ++t) {
        int la = level_of_mag(abs(k1[t]), n_levels, edges);
        int lb = level_of_mag(abs(k2[t]), n_levels, edges);
        if (la == lb) {
            level[t] = la; kind[t] = (la <= n_levels) ? 0 : -1;
        } else if (la < lb) {
            level[t] = la; kind[t] = 1;
        } else {
            level[t] = lb; kind[t] = 2;
        }
        if (level[t] > n_levels) { level[t] = -1; kind[t] = -1; }
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3: local domain of level l centred at macro node X_ij = (iH, jH).     */
/* The patch has n x n nodes with spacing h = L / n on the lattice           */
/* 2*pi*idx / Nl (Nl = 2*pi / h, an integer); its centre is the lattice      */
/* node nearest to X_ij (ties rounded up) and node a sits at lattice index   */
/* centre - n/2 + a.                                                         */
/* ------------------------------------------------------------------------ */
long orc_patch_origin(int i, int n_macro, long Nl, int n)
{
    /* nearest lattice index to i * Nl / n_macro, halves rounded up */
    long c = (2L * (long)i * Nl + (long)n_macro) / (2L * (long)n_macro);
    return c - n / 2;
}

static long pmod(long a, long m) { long r = a % m; return r < 0 ? r + m : r; }

/* psi at lattice indices (gx, gy) of an Nl-point lattice, summed mode by mode */
static double psi_at(int n_modes, const int *k1, const int *k2, const double *re,
                     const double *im, const unsigned char *use, long Nl, long gx, long gy)
{
    double s = 0.0;
    for (int t = 0; t < n_modes; ++t) {
        if (use && !use[t]) continue;
        long r = pmod((long)k1[t] * gx + (long)k2[t] * gy, Nl);   /* exact phase index */
        double th = 2.0 * ORC_PI * (double)r / (double)Nl;
        s += re[t] * cos(th) - im[t] * sin(th);
    }
    return s;
}

/* The selected modes (use[t] != 0, or all with use == NULL) copied in their  */
/* order to a list of their own, so that a synthesis visits only those; the   */
/* sums psi_at forms over the list are the same sums in the same order.       */
typedef struct { int n; int *k1, *k2; double *re, *im; } mode_list;

static mode_list select_modes(int n_modes, const int *k1, const int *k2, const double *re,
                              const double *im, const unsigned char *use)
{
    mode_list m;
    m.n = 0;
    m.k1 = malloc(sizeof(int) * (n_modes + 1)); m.k2 = malloc(sizeof(int) * (n_modes + 1));
    m.re = malloc(sizeof(double) * (n_modes + 1)); m.im = malloc(sizeof(double) * (n_modes + 1));
    for (int t = 0; t < n_modes; ++t) {
        if (use && !use[t]) continue;
        m.k1[m.n] = k1[t]; m.k2[m.n] = k2[t]; m.re[m.n] = re[t]; m.im[m.n] = im[t];
        ++m.n;
    }
    return m;
}

static void free_modes(mode_list *m) { free(m->k1); free(m->k2); free(m->re); free(m->im); }

/* psi of the selected modes on the patch nodes, patch mean removed. */
void orc_patch_psi(int n_modes, const int *k1, const int *k2, const double *re,
                   const double *im, const unsigned char *use, long Nl, long ox, long oy,
                   int n, double *psi)
{
    mode_list md = select_modes(n_modes, k1, k2, re, im, use);
    double mean = 0.0;
    for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
            double p = psi_at(md.n, md.k1, md.k2, md.re, md.im, NULL, Nl, ox + a, oy + b);
            psi[(long)b * n + a] = p;
            mean += p;
        }
    mean /= (double)n * (double)n;
    for (long c = 0; c < (long)n * n; ++c) psi[c] -= mean;
    free_modes(&md);
}

/* Sec. 2.1: v = (-d psi/dx2, d psi/dx1) with central differences; indices  */
/* wrap on the patch (periodic local problem).                               */
void orc_velocity(int n, double h, const double *psi, double *v1, double *v2)
{
    for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
            int ap = (a + 1) % n, am = (a + n - 1) % n;
            int bp = (b + 1) % n, bm = (b + n - 1) % n;
            v1[b * n + a] = -(psi[bp * n + a] - psi[bm * n + a]) / (2.0 * h);
            v2[b * n + a] = (psi[b * n + ap] - psi[b * n + am]) / (2.0 * h);
        }
}

/* smallest eigenvalue of the symmetric 2x2 tensor (B11, B12, B22) */
double orc_lambda_min(const double *B)
{
    double tr = B[0] + B[2];
    double d = sqrt((B[0] - B[2]) * (B[0] - B[2]) + 4.0 * B[1] * B[1]);
    return 0.5 * (tr - d);
}

/* Time step of the micro solver: CFL on advection and on diffusion, and     */
/* never above the RK2 + central-advection stability bound                   */
/* (8 lambda_min h^2 / vmax^4)^(1/3).  vmax = max(|v1| + |v2|).              */
double orc_micro_dt(double h, double vmax, const double *B, double cfl)
{
    double dd = h * h / (2.0 * (B[0] + B[2]) + 4.0 * fabs(B[1]));
    double dt = dd;
    if (vmax > 0.0) {
        double da = h / vmax;
        if (da < dt) dt = da;
    }
    dt *= cfl;
    if (vmax > 0.0) {
        double ds = cbrt(8.0 * orc_lambda_min(B) * h * h / (vmax * vmax * vmax * vmax));
        if (ds < dt) dt = ds;
    }
    return dt;
}

/* Quasi-stationarity window: relaxation time tau = L^2 / (4 pi^2 lambda_min)*/
/* of the slowest patch mode; burn-in t_burn * tau, averaging t_avg * tau.   */
void orc_micro_steps(double L, const double *B, double dt, double t_burn, double t_avg,
                     long *n_burn, long *n_avg)
{
    double tau = L * L / (4.0 * ORC_PI * ORC_PI * orc_lambda_min(B));
    *n_burn = (long)ceil(t_burn * tau / dt);
    *n_avg = (long)ceil(t_avg * tau / dt);
    if (*n_avg < 1) *n_avg = 1;
}

/* right-hand side f_j(w) of the corrector equation for gradient e_j         */
static void corrector_rhs(int n, double h, const double *v1, const double *v2,
                          const double *B, int j, const double *w, double *f)
{
    double g1 = (j == 1) ? 1.0 : 0.0, g2 = (j == 2) ? 1.0 : 0.0;
    for (int b = 0; b < n; ++b) {
        int bp = (b + 1) % n, bm = (b + n - 1) % n;
        for (int a = 0; a < n; ++a) {
            int ap = (a + 1) % n, am = (a + n - 1) % n;
            double wc = w[b * n + a];
            double d0x = (w[b * n + ap] - w[b * n + am]) / (2.0 * h);
            double d0y = (w[bp * n + a] - w[bm * n + a]) / (2.0 * h);
            double dxx = (w[b * n + ap] - 2.0 * wc + w[b * n + am]) / (h * h);
            double dyy = (w[bp * n + a] - 2.0 * wc + w[bm * n + a]) / (h * h);
            double dxy = (w[bp * n + ap] - w[bp * n + am] - w[bm * n + ap] + w[bm * n + am])
                         / (4.0 * h * h);
            f[b * n + a] = v1[b * n + a] * (d0x + g1) + v2[b * n + a] * (d0y + g2)
                         + B[0] * dxx + 2.0 * B[1] * dxy + B[2] * dyy;
        }
    }
}

/* Exposed for the brute-force steady-state test: f_j(w) on a patch. */
void orc_corrector_rhs(int n, double h, const double *psi, const double *B, int j,
                       const double *w, double *f)
{
    double *v1 = malloc(sizeof(double) * n * n), *v2 = malloc(sizeof(double) * n * n);
    orc_velocity(n, h, psi, v1, v2);
    corrector_rhs(n, h, v1, v2, B, j, w, f);
    free(v1); free(v2);
}

/* ------------------------------------------------------------------------ */
/* Energy form of the corrector pair (the other side of HMM step 3's flux    */
/* average): for the periodic fields w[2][n][n] and the base B,              */
/*   E_jk = mean over nodes of  B11 (D+x w_j)(D+x w_k)                       */
/*          + B12 ((D0x w_j)(D0y w_k) + (D0y w_j)(D0x w_k))                  */
/*          + B22 (D+y w_j)(D+y w_k),                                        */
/* D+ forward, D0 central differences; and mass[j] = mean of w_j.  These are */
/* the forms that summation by parts gives for the stencil of orc_corrector_ */
/* rhs: at the steady state E = K - B up to the O(h^2) remainder of the      */
/* central advection term (exactly for shear flows).                         */
/* ------------------------------------------------------------------------ */
void orc_corrector_energy(int n, double h, const double *w, const double *B, double *E,
                          double *mass)
{
    const double *w1 = w, *w2 = w + (long)n * n;
    double e11 = 0.0, e12 = 0.0, e22 = 0.0, m1 = 0.0, m2 = 0.0;
    for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
            const int ap = (a + 1) % n, am = (a + n - 1) % n, bp = (b + 1) % n, bm = (b + n - 1) % n;
#define W(f, x, y) f[(long)(y) * n + (x)]
            const double fx1 = (W(w1, ap, b) - W(w1, a, b)) / h, fy1 = (W(w1, a, bp) - W(w1, a, b)) / h;
            const double fx2 = (W(w2, ap, b) - W(w2, a, b)) / h, fy2 = (W(w2, a, bp) - W(w2, a, b)) / h;
            const double cx1 = (W(w1, ap, b) - W(w1, am, b)) / (2.0 * h);
            const double cy1 = (W(w1, a, bp) - W(w1, a, bm)) / (2.0 * h);
            const double cx2 = (W(w2, ap, b) - W(w2, am, b)) / (2.0 * h);
            const double cy2 = (W(w2, a, bp) - W(w2, a, bm)) / (2.0 * h);
            m1 += W(w1, a, b);
            m2 += W(w2, a, b);
#undef W
            e11 += B[0] * fx1 * fx1 + 2.0 * B[1] * cx1 * cy1 + B[2] * fy1 * fy1;
            e12 += B[0] * fx1 * fx2 + B[1] * (cx1 * cy2 + cy1 * cx2) + B[2] * fy1 * fy2;
            e22 += B[0] * fx2 * fx2 + 2.0 * B[1] * cx2 * cy2 + B[2] * fy2 * fy2;
        }
    const double nn = (double)n * n;
    E[0] = e11 / nn; E[1] = e12 / nn; E[2] = e22 / nn;
    if (mass) { mass[0] = m1 / nn; mass[1] = m2 / nn; }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2 (HMM steps 1-3) and the K[psi, B; D] notation of Sec. 2.2:       */
/* for each gradient G = e_j the reconstruction is u = G.x + w with w        */
/* periodic on the patch, w(0) = 0; w is advanced with Heun's RK2 for        */
/* n_burn + n_avg steps; after each of the last n_avg steps the spatial mean */
/* of v_i w_j is added to S_ij.  The effective flux for G = e_j is           */
/* P_j = B e_j + S_.j / n_avg, and K is its symmetric part:                  */
/*   K11 = P_1,1   K22 = P_2,2   K12 = (P_1,2 + P_2,1) / 2.                  */
/* Optional outputs: w_out[2][n][n] (final corrector fields), S_out[4] =     */
/* time-averaged (S11, S21, S12, S22).                                       */
/* ------------------------------------------------------------------------ */
void orc_patch_k(int n, double h, const double *psi, const double *B, double dt,
                 long n_burn, long n_avg, double *K, double *w_out, double *S_out)
{
    long nn = (long)n * n;
    double *v1 = malloc(sizeof(double) * nn), *v2 = malloc(sizeof(double) * nn);
    double *w = malloc(sizeof(double) * nn), *ws = malloc(sizeof(double) * nn);
    double *f = malloc(sizeof(double) * nn);
    double S[2][2] = {{0, 0}, {0, 0}};          /* S[i][j] = sum of mean(v_i w_j) */
    orc_velocity(n, h, psi, v1, v2);
    for (int j = 1; j <= 2; ++j) {
        memset(w, 0, sizeof(double) * nn);
        for (long s = 1; s <= n_burn + n_avg; ++s) {
            corrector_rhs(n, h, v1, v2, B, j, w, f);
            for (long c = 0; c < nn; ++c) ws[c] = w[c] + dt * f[c];
            corrector_rhs(n, h, v1, v2, B, j, ws, f);
            for (long c = 0; c < nn; ++c) w[c] = 0.5 * (w[c] + ws[c] + dt * f[c]);
            if (s > n_burn) {
                double m1 = 0.0, m2 = 0.0;
                for (long c = 0; c < nn; ++c) { m1 += v1[c] * w[c]; m2 += v2[c] * w[c]; }
                S[0][j - 1] += m1 / (double)nn;
                S[1][j - 1] += m2 / (double)nn;
            }
        }
        if (w_out) memcpy(w_out + (j - 1) * nn, w, sizeof(double) * nn);
    }
    double P11 = B[0] + S[0][0] / (double)n_avg;   /* P_1 = B e_1 + S_.1 */
    double P21 = B[1] + S[1][0] / (double)n_avg;
    double P12 = B[1] + S[0][1] / (double)n_avg;   /* P_2 = B e_2 + S_.2 */
    double P22 = B[2] + S[1][1] / (double)n_avg;
    K[0] = P11;
    K[1] = 0.5 * (P21 + P12);
    K[2] = P22;
    if (S_out) {
        S_out[0] = S[0][0] / n_avg; S_out[1] = S[1][0] / n_avg;
        S_out[2] = S[0][1] / n_avg; S_out[3] = S[1][1] / n_avg;
    }
    free(v1); free(v2); free(w); free(ws); free(f);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (per off-diagonal part): treat psi_12 (fine in x2) as a shear */
/* on every patch column x1 = x_a and psi_21 (fine in x1) as a shear on      */
/* every patch row x2 = x_b.  q is the line variance of the part, sampled at */
/* r points per patch cell along the line, r = ceil(10 kmax L / (2 pi n)):   */
/*   q12[a] = mean_s (psi12(x_a, y_s) - mean)^2,                             */
/*   q21[b] = mean_s (psi21(x_s, y_b) - mean)^2.                             */
/* Inputs: the level's mode list with part flags (kind 1 or 2).             */
/* ------------------------------------------------------------------------ */
static int line_refine(int n_modes, const int *kx, const unsigned char *use, double L, int n)
{
    int kmax = 0;
    for (int t = 0; t < n_modes; ++t)
        if (use[t] && abs(kx[t]) > kmax) kmax = abs(kx[t]);
    double need = 10.0 * kmax * L / (2.0 * ORC_PI);
    int r = (int)ceil(need / (double)n);
    return r < 1 ? 1 : r;
}

void orc_offdiag_q(int n_modes, const int *k1, const int *k2, const double *re,
                   const double *im, const unsigned char *use12, const unsigned char *use21,
                   long Nl, long ox, long oy, int n, double L, double *q12, double *q21)
{
    int r12 = line_refine(n_modes, k2, use12, L, n);
    int r21 = line_refine(n_modes, k1, use21, L, n);
    int any12 = 0, any21 = 0;
    for (int t = 0; t < n_modes; ++t) { any12 |= use12[t]; any21 |= use21[t]; }
    mode_list m12 = select_modes(n_modes, k1, k2, re, im, use12);
    mode_list m21 = select_modes(n_modes, k1, k2, re, im, use21);
    /* columns and rows are independent; the threads split them (a team only  */
    /* where no enclosing parallel region is active, e.g. a one-node chain)    */
#pragma omp parallel for schedule(dynamic, 1)
    for (int a = 0; a < n; ++a) {
        q12[a] = 0.0;
        if (!any12) continue;
        /* column x_a = lattice index ox + a on the Nl lattice, i.e. index     */
        /* (ox + a) * r12 on the refined lattice of Nl * r12 points; samples   */
        /* y_s at refined indices oy * r12 + s, s = 0 .. n * r12 - 1           */
        long m = (long)n * r12, Nr = Nl * r12;
        double mean = 0.0, sq = 0.0;
        double *g = malloc(sizeof(double) * m);
        for (long s = 0; s < m; ++s) {
            g[s] = psi_at(m12.n, m12.k1, m12.k2, m12.re, m12.im, NULL, Nr, (ox + a) * (long)r12,
                          oy * r12 + s);
            mean += g[s];
        }
        mean /= (double)m;
        for (long s = 0; s < m; ++s) sq += (g[s] - mean) * (g[s] - mean);
        q12[a] = sq / (double)m;
        free(g);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < n; ++b) {
        q21[b] = 0.0;
        if (!any21) continue;
        long m = (long)n * r21, Nr = Nl * r21;
        double mean = 0.0, sq = 0.0;
        double *g = malloc(sizeof(double) * m);
        for (long s = 0; s < m; ++s) {
            g[s] = psi_at(m21.n, m21.k1, m21.k2, m21.re, m21.im, NULL, Nr, ox * r21 + s,
                          (oy + b) * (long)r21);
            mean += g[s];
        }
        mean /= (double)m;
        for (long s = 0; s < m; ++s) sq += (g[s] - mean) * (g[s] - mean);
        q21[b] = sq / (double)m;
        free(g);
    }
    free_modes(&m12);
    free_modes(&m21);
}

/* Algorithms 1 and 2 given the line variances:                             */
/*   psi_12: K*11(x_a) = B11 + q12[a] / B22 (Eq. shearhomoY), then the      */
/*           layered-medium harmonic mean across the columns;               */
/*   psi_21: K*22(x_b) = B22 + q21[b] / B11 (Eq. shearhomoX), harmonic mean */
/*           across the rows;                                               */
/*   K_off = K[psi_12; B] + K[psi_21; B] - B.                               */
/* B12 and the component along the layers pass through unchanged.  A part   */
/* the level does not have (q array NULL) contributes K[0; B] = B exactly.  */
void orc_offdiag_apply(int n, const double *q12, const double *q21, const double *B,
                       double *Koff)
{
    double K12_11 = B[0], K21_22 = B[2];   /* K[psi_12; B] = [[K12_11, B12], [B12, B22]] */
    if (q12) {                              /* K[psi_21; B] = [[B11, B12], [B12, K21_22]] */
        double s1 = 0.0;
        for (int a = 0; a < n; ++a) s1 += 1.0 / (B[0] + q12[a] / B[2]);
        K12_11 = (double)n / s1;
    }
    if (q21) {
        double s2 = 0.0;
        for (int b = 0; b < n; ++b) s2 += 1.0 / (B[2] + q21[b] / B[0]);
        K21_22 = (double)n / s2;
    }
    if (!q12 && !q21) { memcpy(Koff, B, sizeof(double) * 3); return; }
    Koff[0] = K12_11 + B[0] - B[0];
    Koff[1] = B[1] + B[1] - B[1];
    Koff[2] = B[2] + K21_22 - B[2];
}

/* ------------------------------------------------------------------------ */
/* Patch resolution rule for uneven patch sizes: at least 10 points per      */
/* wavelength of the level's finest diagonal mode and a cell Peclet number   */
/* of at most 2 with the molecular diffusivity (the smallest base the level  */
/* can see):  n = clamp(pow2ceil(max(10 kmax L / 2pi, L vmax / (2 kappa))),  */
/* n_min, n_max).  kmax = max(|k1|, |k2|) over the level's diagonal modes;   */
/* vmax = max |v| of the band's exact velocity                              */
/*   v1 = sum k2 (re sin t + im cos t),  v2 = -sum k1 (re sin t + im cos t)  */
/* over the patch's nodes on a reference grid of nref x nref points.        */
/* ------------------------------------------------------------------------ */
int orc_patch_n_rule(int n_modes, const int *k1, const int *k2, const double *re,
                     const double *im, const unsigned char *use, long m, int i, int j,
                     int n_macro, double kappa, int nref, int n_min, int n_max, double *vmax_out)
{
    int kmax = 0;
    for (int t = 0; t < n_modes; ++t)
        if (use[t]) {
            int a = abs(k1[t]) > abs(k2[t]) ? abs(k1[t]) : abs(k2[t]);
            if (a > kmax) kmax = a;
        }
    long Nr = (long)nref * m;
    long ox = orc_patch_origin(i, n_macro, Nr, nref), oy = orc_patch_origin(j, n_macro, Nr, nref);
    double vmax = 0.0;
    for (int b = 0; b < nref; ++b)
        for (int a = 0; a < nref; ++a) {
            double v1 = 0.0, v2 = 0.0;
            for (int t = 0; t < n_modes; ++t) {
                if (!use[t]) continue;
                long r = pmod((long)k1[t] * (ox + a) + (long)k2[t] * (oy + b), Nr);
                double th = 2.0 * ORC_PI * (double)r / (double)Nr;
                double q = re[t] * sin(th) + im[t] * cos(th);
                v1 += k2[t] * q;
                v2 -= k1[t] * q;
            }
            double sp = sqrt(v1 * v1 + v2 * v2);
            if (sp > vmax) vmax = sp;
        }
    if (vmax_out) *vmax_out = vmax;
    double L = 2.0 * ORC_PI / (double)m;
    double need = 10.0 * kmax * L / (2.0 * ORC_PI);
    double pe = L * vmax / (2.0 * kappa);
    if (pe > need) need = pe;
    int n = n_min;
    while (n < n_max && (double)n < need) n *= 2;
    return n;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 3, applied recursively from the finest level (L) to the        */
/* coarsest (1), for a set of macro nodes:                                   */
/*   B_1 = kappa I;  Koff_l = K_off,l(B_l);  B_{l+1} = Koff_l   (top-down)  */
/*   K*_L = K[psi_L,diag ; K_off,L(B_L)]                                    */
/*   for l = L-1 .. 1:  Knet = K*_{l+1} - Koff_l + B_l                      */
/*                      K*_l = K[psi_l,diag ; K_off,l(Knet)]                */
/*   K = K*_1                                                               */
/* psi_l,diag is the diagonal band of level l; K_off,l is Algorithms 1-2     */
/* with level l's off-diagonal parts (the identity when there are none).    */
/* Patch geometry: level l has side L_l = 2 pi / patch_div[l]; the patch of  */
/* node p at level l has node_n[p * L + l] points per side (lattice          */
/* Nl = n * patch_div[l]).                                                  */
/* Outputs per node: K[3] and, optionally, the per-level K*_l [L][3] and the  */
/* step counts n_burn + n_avg of every level's patch solve [L].              */
/* The time step and window of every patch solve follow orc_micro_dt and    */
/* orc_micro_steps, unless n_burn_fixed / n_avg_fixed are positive.         */
/* ------------------------------------------------------------------------ */
void orc_chain(int n_modes, const int *k1, const int *k2, const double *re, const double *im,
               int n_levels, const double *edges, const int *node_n, const long *patch_div,
               int n_macro, double kappa, double cfl, double t_burn, double t_avg,
               long n_burn_fixed, long n_avg_fixed,
               int n_nodes, const int *node_i, const int *node_j,
               double *K_out, double *Kstar_levels_out, long *steps_out, int periodize)
{
    int *lev = malloc(sizeof(int) * n_modes), *kind = malloc(sizeof(int) * n_modes);
    orc_band_of(n_modes, k1, k2, n_levels, edges, lev, kind);

#pragma omp parallel for schedule(dynamic, 1) if (n_nodes > 1)
    for (int p = 0; p < n_nodes; ++p) {
        unsigned char *ud = malloc(n_modes), *u12 = malloc(n_modes), *u21 = malloc(n_modes);
        double (*Bl)[3] = malloc(sizeof(double) * 3 * (n_levels + 2));
        double (*Koffl)[3] = malloc(sizeof(double) * 3 * (n_levels + 2));
        double Kstar[3], base[3], Knet[3];
        int nmax = 0;
        for (int l = 0; l < n_levels; ++l) if (node_n[(long)p * n_levels + l] > nmax) nmax = node_n[(long)p * n_levels + l];
        double *psi = malloc(sizeof(double) * nmax * nmax);
        double **Q12 = malloc(sizeof(double *) * n_levels), **Q21 = malloc(sizeof(double *) * n_levels);

        /* per level: line variances of the off-diagonal parts at this node */
        for (int l = 1; l <= n_levels; ++l) {
            int n = node_n[(long)p * n_levels + (l - 1)];
            long Nl = (long)n * patch_div[l - 1];
            long ox = orc_patch_origin(node_i[p], n_macro, Nl, n);
            long oy = orc_patch_origin(node_j[p], n_macro, Nl, n);
            double L = 2.0 * ORC_PI * n / (double)Nl;
            for (int t = 0; t < n_modes; ++t) {
                u12[t] = (lev[t] == l && kind[t] == 1);
                u21[t] = (lev[t] == l && kind[t] == 2);
            }
            int any12 = 0, any21 = 0;
            for (int t = 0; t < n_modes; ++t) { any12 |= u12[t]; any21 |= u21[t]; }
            Q12[l - 1] = malloc(sizeof(double) * n);
            Q21[l - 1] = malloc(sizeof(double) * n);
            orc_offdiag_q(n_modes, k1, k2, re, im, u12, u21, Nl, ox, oy, n, L,
                          Q12[l - 1], Q21[l - 1]);
            if (!any12) { free(Q12[l - 1]); Q12[l - 1] = NULL; }
            if (!any21) { free(Q21[l - 1]); Q21[l - 1] = NULL; }
        }
        /* top-down closed forms */
        Bl[1][0] = kappa; Bl[1][1] = 0.0; Bl[1][2] = kappa;
        for (int l = 1; l <= n_levels; ++l) {
            orc_offdiag_apply(node_n[(long)p * n_levels + (l - 1)], Q12[l - 1], Q21[l - 1], Bl[l], Koffl[l]);
            if (l < n_levels) memcpy(Bl[l + 1], Koffl[l], sizeof(double) * 3);
        }
        /* bottom-up patch solves */
        for (int l = n_levels; l >= 1; --l) {
            int n = node_n[(long)p * n_levels + (l - 1)];
            long Nl = (long)n * patch_div[l - 1];
            long ox = orc_patch_origin(node_i[p], n_macro, Nl, n);
            long oy = orc_patch_origin(node_j[p], n_macro, Nl, n);
            double L = 2.0 * ORC_PI * n / (double)Nl;
            double h = L / n;
            if (l == n_levels) {
                memcpy(base, Koffl[l], sizeof(base));
            } else {
                for (int c = 0; c < 3; ++c) Knet[c] = Kstar[c] - Koffl[l][c] + Bl[l][c];
                orc_offdiag_apply(n, Q12[l - 1], Q21[l - 1], Knet, base);
            }
            for (int t = 0; t < n_modes; ++t) ud[t] = (lev[t] == l && kind[t] == 0);
            orc_patch_psi(n_modes, k1, k2, re, im, ud, Nl, ox, oy, n, psi);
            if (periodize) {              /* the band's periodic component on the patch */
                double *pp = malloc(sizeof(double) * n * n);
                orc_periodic_smooth(n, psi, pp);
                memcpy(psi, pp, sizeof(double) * n * n);
                free(pp);
            }
            double *v1 = malloc(sizeof(double) * n * n), *v2 = malloc(sizeof(double) * n * n);
            orc_velocity(n, h, psi, v1, v2);
            double vmax = 0.0;
            for (long c = 0; c < (long)n * n; ++c) {
                double s = fabs(v1[c]) + fabs(v2[c]);
                if (s > vmax) vmax = s;
            }
            free(v1); free(v2);
            double dt = orc_micro_dt(h, vmax, base, cfl);
            long nb, na;
            orc_micro_steps(L, base, dt, t_burn, t_avg, &nb, &na);
            if (n_burn_fixed >= 0 && n_avg_fixed > 0) { nb = n_burn_fixed; na = n_avg_fixed; }
            if (steps_out) steps_out[(long)p * n_levels + (l - 1)] = nb + na;
            orc_patch_k(n, h, psi, base, dt, nb, na, Kstar, NULL, NULL);
            if (Kstar_levels_out)
                memcpy(Kstar_levels_out + ((long)p * n_levels + (l - 1)) * 3, Kstar,
                       sizeof(double) * 3);
        }
        memcpy(K_out + (long)p * 3, Kstar, sizeof(double) * 3);
        for (int l = 0; l < n_levels; ++l) { free(Q12[l]); free(Q21[l]); }
        free(Q12); free(Q21); free(psi);
        free(ud); free(u12); free(u21); free(Bl); free(Koffl);
    }
    free(lev); free(kind);
}

/* ------------------------------------------------------------------------ */
/* Macro solver for Eq. (homo): U_t = div(K grad U) on the periodic N x N    */
/* node grid (spacing H = 2 pi / N), conservative form with face tensors     */
/* K_f = (K_node + K_neighbour) / 2:                                         */
/*   Fx(i+1/2,j) = K11f (U(i+1,j) - U(i,j)) / H                              */
/*              + K12f (U(i,j+1) + U(i+1,j+1) - U(i,j-1) - U(i+1,j-1)) / (4H)*/
/*   Fy(i,j+1/2) = K22f (U(i,j+1) - U(i,j)) / H                              */
/*              + K12f (U(i+1,j) + U(i+1,j+1) - U(i-1,j) - U(i-1,j+1)) / (4H)*/
/*   U_t = (Fx(i+1/2) - Fx(i-1/2) + Fy(j+1/2) - Fy(j-1/2)) / H               */
/* advanced with Heun's RK2.  K is [N*N][3] in node order j*N + i.           */
/* mass_out (nsteps + 1 values or NULL) receives sum(U) * H^2 per step.      */
/* ------------------------------------------------------------------------ */
static void macro_rhs(int N, double H, const double *K, const double *U, double *R)
{
    for (int j = 0; j < N; ++j) {
        int jp = (j + 1) % N, jm = (j + N - 1) % N;
        for (int i = 0; i < N; ++i) {
            int ip = (i + 1) % N, im_ = (i + N - 1) % N;
            /* east face (i+1/2, j) and west face (i-1/2, j) */
            double fe, fw, fn, fs;
            {
                const double *a = K + 3L * (j * N + i), *b = K + 3L * (j * N + ip);
                double k11 = 0.5 * (a[0] + b[0]), k12 = 0.5 * (a[1] + b[1]);
                fe = k11 * (U[j * N + ip] - U[j * N + i]) / H
                   + k12 * (U[jp * N + i] + U[jp * N + ip] - U[jm * N + i] - U[jm * N + ip]) / (4.0 * H);
            }
            {
                const double *a = K + 3L * (j * N + im_), *b = K + 3L * (j * N + i);
                double k11 = 0.5 * (a[0] + b[0]), k12 = 0.5 * (a[1] + b[1]);
                fw = k11 * (U[j * N + i] - U[j * N + im_]) / H
                   + k12 * (U[jp * N + im_] + U[jp * N + i] - U[jm * N + im_] - U[jm * N + i]) / (4.0 * H);
            }
            {
                const double *a = K + 3L * (j * N + i), *b = K + 3L * (jp * N + i);
                double k22 = 0.5 * (a[2] + b[2]), k12 = 0.5 * (a[1] + b[1]);
                fn = k22 * (U[jp * N + i] - U[j * N + i]) / H
                   + k12 * (U[j * N + ip] + U[jp * N + ip] - U[j * N + im_] - U[jp * N + im_]) / (4.0 * H);
            }
            {
                const double *a = K + 3L * (jm * N + i), *b = K + 3L * (j * N + i);
                double k22 = 0.5 * (a[2] + b[2]), k12 = 0.5 * (a[1] + b[1]);
                fs = k22 * (U[j * N + i] - U[jm * N + i]) / H
                   + k12 * (U[jm * N + ip] + U[j * N + ip] - U[jm * N + im_] - U[j * N + im_]) / (4.0 * H);
            }
            R[j * N + i] = (fe - fw + fn - fs) / H;
        }
    }
}

/* dt = cfl * H^2 / max_nodes(K11 + K22 + |K12|) */
double orc_macro_dt(int N, const double *K, double cfl)
{
    double H = 2.0 * ORC_PI / N, m = 0.0;
    for (long p = 0; p < (long)N * N; ++p) {
        double s = K[3 * p] + K[3 * p + 2] + fabs(K[3 * p + 1]);
        if (s > m) m = s;
    }
    return cfl * H * H / m;
}

void orc_macro_run(int N, double *U, const double *K, double dt, long nsteps, double *mass_out)
{
    double H = 2.0 * ORC_PI / N;
    long nn = (long)N * N;
    double *R = malloc(sizeof(double) * nn), *Us = malloc(sizeof(double) * nn);
    if (mass_out) { double m = 0; for (long c = 0; c < nn; ++c) m += U[c]; mass_out[0] = m * H * H; }
    for (long s = 1; s <= nsteps; ++s) {
        macro_rhs(N, H, K, U, R);
        for (long c = 0; c < nn; ++c) Us[c] = U[c] + dt * R[c];
        macro_rhs(N, H, K, Us, R);
        for (long c = 0; c < nn; ++c) U[c] = 0.5 * (U[c] + Us[c] + dt * R[c]);
        if (mass_out) { double m = 0; for (long c = 0; c < nn; ++c) m += U[c]; mass_out[s] = m * H * H; }
    }
    free(R); free(Us);
}

/* ------------------------------------------------------------------------ */
/* Direct simulation of Eq. (model), u_t = v.grad u + kappa Lap u, on the    */
/* full Nf x Nf grid with the same second-order central differences and      */
/* Heun's RK2 as the local problems (the Sec. 4 reference scheme: second     */
/* order in space and time).  psi is the stream function on the grid.       */
/* ------------------------------------------------------------------------ */
static void dns_rhs(int Nf, double h, const double *v1, const double *v2, double kappa,
                    const double *u, double *f)
{
#pragma omp parallel for
    for (int b = 0; b < Nf; ++b) {
        int bp = (b + 1) % Nf, bm = (b + Nf - 1) % Nf;
        for (int a = 0; a < Nf; ++a) {
            int ap = (a + 1) % Nf, am = (a + Nf - 1) % Nf;
            long c = (long)b * Nf + a;
            double uc = u[c];
            double d0x = (u[(long)b * Nf + ap] - u[(long)b * Nf + am]) / (2.0 * h);
            double d0y = (u[(long)bp * Nf + a] - u[(long)bm * Nf + a]) / (2.0 * h);
            double lap = (u[(long)b * Nf + ap] + u[(long)b * Nf + am] + u[(long)bp * Nf + a]
                          + u[(long)bm * Nf + a] - 4.0 * uc) / (h * h);
            f[c] = v1[c] * d0x + v2[c] * d0y + kappa * lap;
        }
    }
}

void orc_dns_run(int Nf, const double *psi, double kappa, double dt, long nsteps, double *u)
{
    long nn = (long)Nf * Nf;
    double h = 2.0 * ORC_PI / Nf;
    double *v1 = malloc(sizeof(double) * nn), *v2 = malloc(sizeof(double) * nn);
    double *f = malloc(sizeof(double) * nn), *us = malloc(sizeof(double) * nn);
    orc_velocity(Nf, h, psi, v1, v2);
    for (long s = 0; s < nsteps; ++s) {
        dns_rhs(Nf, h, v1, v2, kappa, u, f);
        for (long c = 0; c < nn; ++c) us[c] = u[c] + dt * f[c];
        dns_rhs(Nf, h, v1, v2, kappa, us, f);
        for (long c = 0; c < nn; ++c) u[c] = 0.5 * (u[c] + us[c] + dt * f[c]);
    }
    free(v1); free(v2); free(f); free(us);
}

/* ------------------------------------------------------------------------ */
/* Sec. 4 set-up: Dirichlet conditions in x1, periodic in x2.  The paper     */
/* solves on [0,1]^2 with u = 1 at x1 = 0, u = 0 at x1 = 1 and the step      */
/* u0 = 1 for x1 <= 1/2, else 0.  Here the same problem is posed on          */
/* [0, 2 pi] x [0, 2 pi): nodes x1 = i H (H = 2 pi / N), column i = 0 is the  */
/* boundary x1 = 0 (held at u_left) and a virtual column i = N is the        */
/* boundary x1 = 2 pi (value u_right); columns 1..N-1 are the unknowns.  The */
/* K field (or the velocity) is periodic, so its column N is its column 0.   */
/* The interior scheme is the periodic one unchanged.                        */
/* ------------------------------------------------------------------------ */
static double u_dir(const double *U, int N, int i, int j, double u_right)
{
    return i == N ? u_right : U[(long)j * N + i];
}

static void macro_rhs_dir(int N, double H, const double *K, const double *U, double ur, double *R)
{
#pragma omp parallel for
    for (int j = 0; j < N; ++j) {
        int jp = (j + 1) % N, jm = (j + N - 1) % N;
        R[(long)j * N] = 0.0;
        for (int i = 1; i < N; ++i) {
            int ip = i + 1, im_ = i - 1, ipk = ip % N;
            double fe, fw, fn, fs;
            {
                const double *a = K + 3L * (j * N + i), *b = K + 3L * (j * N + ipk);
                double k11 = 0.5 * (a[0] + b[0]), k12 = 0.5 * (a[1] + b[1]);
                fe = k11 * (u_dir(U, N, ip, j, ur) - u_dir(U, N, i, j, ur)) / H
                   + k12 * (u_dir(U, N, i, jp, ur) + u_dir(U, N, ip, jp, ur)
                            - u_dir(U, N, i, jm, ur) - u_dir(U, N, ip, jm, ur)) / (4.0 * H);
            }
            {
                const double *a = K + 3L * (j * N + im_), *b = K + 3L * (j * N + i);
                double k11 = 0.5 * (a[0] + b[0]), k12 = 0.5 * (a[1] + b[1]);
                fw = k11 * (u_dir(U, N, i, j, ur) - u_dir(U, N, im_, j, ur)) / H
                   + k12 * (u_dir(U, N, im_, jp, ur) + u_dir(U, N, i, jp, ur)
                            - u_dir(U, N, im_, jm, ur) - u_dir(U, N, i, jm, ur)) / (4.0 * H);
            }
            {
                const double *a = K + 3L * (j * N + i), *b = K + 3L * (jp * N + i);
                double k22 = 0.5 * (a[2] + b[2]), k12 = 0.5 * (a[1] + b[1]);
                fn = k22 * (u_dir(U, N, i, jp, ur) - u_dir(U, N, i, j, ur)) / H
                   + k12 * (u_dir(U, N, ip, j, ur) + u_dir(U, N, ip, jp, ur)
                            - u_dir(U, N, im_, j, ur) - u_dir(U, N, im_, jp, ur)) / (4.0 * H);
            }
            {
                const double *a = K + 3L * (jm * N + i), *b = K + 3L * (j * N + i);
                double k22 = 0.5 * (a[2] + b[2]), k12 = 0.5 * (a[1] + b[1]);
                fs = k22 * (u_dir(U, N, i, j, ur) - u_dir(U, N, i, jm, ur)) / H
                   + k12 * (u_dir(U, N, ip, jm, ur) + u_dir(U, N, ip, j, ur)
                            - u_dir(U, N, im_, jm, ur) - u_dir(U, N, im_, j, ur)) / (4.0 * H);
            }
            R[(long)j * N + i] = (fe - fw + fn - fs) / H;
        }
    }
}

/* Heun steps of the macro problem with the Dirichlet x1 boundaries; column 0 */
/* of U is set to u_left first and stays there.                              */
void orc_macro_run_dirichlet(int N, double *U, const double *K, double dt, long nsteps,
                             double u_left, double u_right)
{
    double H = 2.0 * ORC_PI / N;
    long nn = (long)N * N;
    double *R = malloc(sizeof(double) * nn), *Us = malloc(sizeof(double) * nn);
    for (int j = 0; j < N; ++j) U[(long)j * N] = u_left;
    for (long s = 1; s <= nsteps; ++s) {
        macro_rhs_dir(N, H, K, U, u_right, R);
        for (long c = 0; c < nn; ++c) Us[c] = U[c] + dt * R[c];
        macro_rhs_dir(N, H, K, Us, u_right, R);
        for (long c = 0; c < nn; ++c) U[c] = 0.5 * (U[c] + Us[c] + dt * R[c]);
    }
    free(R); free(Us);
}

/* The direct simulation of the Sec. 4 set-up: the DNS scheme of             */
/* orc_dns_run on the interior columns 1..Nf-1, column 0 held at u_left and  */
/* the virtual column Nf at u_right.                                         */
static void dns_rhs_dir(int Nf, double h, const double *v1, const double *v2, double kappa,
                        const double *u, double ur, double *f)
{
#pragma omp parallel for
    for (int b = 0; b < Nf; ++b) {
        int bp = (b + 1) % Nf, bm = (b + Nf - 1) % Nf;
        f[(long)b * Nf] = 0.0;
        for (int a = 1; a < Nf; ++a) {
            long c = (long)b * Nf + a;
            double uc = u[c];
            double ue = u_dir(u, Nf, a + 1, b, ur), uw = u[c - 1];
            double un = u[(long)bp * Nf + a], us = u[(long)bm * Nf + a];
            double d0x = (ue - uw) / (2.0 * h);
            double d0y = (un - us) / (2.0 * h);
            double lap = (ue + uw + un + us - 4.0 * uc) / (h * h);
            f[c] = v1[c] * d0x + v2[c] * d0y + kappa * lap;
        }
    }
}

void orc_dns_run_dirichlet(int Nf, const double *psi, double kappa, double dt, long nsteps,
                           double u_left, double u_right, double *u)
{
    long nn = (long)Nf * Nf;
    double h = 2.0 * ORC_PI / Nf;
    double *v1 = malloc(sizeof(double) * nn), *v2 = malloc(sizeof(double) * nn);
    double *f = malloc(sizeof(double) * nn), *us = malloc(sizeof(double) * nn);
    orc_velocity(Nf, h, psi, v1, v2);
    for (int b = 0; b < Nf; ++b) u[(long)b * Nf] = u_left;
    for (long s = 0; s < nsteps; ++s) {
        dns_rhs_dir(Nf, h, v1, v2, kappa, u, u_right, f);
        for (long c = 0; c < nn; ++c) us[c] = u[c] + dt * f[c];
        dns_rhs_dir(Nf, h, v1, v2, kappa, us, u_right, f);
        for (long c = 0; c < nn; ++c) u[c] = 0.5 * (u[c] + us[c] + dt * f[c]);
    }
    free(v1); free(v2); free(f); free(us);
}

/* stream function of the given modes on the full Nf x Nf grid */
void orc_grid_psi(int n_modes, const int *k1, const int *k2, const double *re,
                  const double *im, int Nf, double *psi)
{
#pragma omp parallel for
    for (int b = 0; b < Nf; ++b)
        for (int a = 0; a < Nf; ++a)
            psi[(long)b * Nf + a] = psi_at(n_modes, k1, k2, re, im, NULL, Nf, a, b);
}

/* box average of the fine field onto the macro grid: macro node (i, j)      */
/* averages the r x r fine nodes with indices i*r - r/2 .. i*r + r/2 - 1     */
/* (periodic), r = Nf / N.  mass = sum over the fine grid of u * h^2.        */
void orc_coarse_grain(int Nf, const double *u, int N, double *U, double *mass)
{
    int r = Nf / N;
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
            double s = 0.0;
            for (int db = 0; db < r; ++db)
                for (int da = 0; da < r; ++da) {
                    long b = pmod((long)j * r - r / 2 + db, Nf), a = pmod((long)i * r - r / 2 + da, Nf);
                    s += u[b * Nf + a];
                }
            U[j * N + i] = s / ((double)r * r);
        }
    if (mass) {
        double h = 2.0 * ORC_PI / Nf, m = 0.0;
        for (long c = 0; c < (long)Nf * Nf; ++c) m += u[c];
        *mass = m * h * h;
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Perturbation moments of the steady corrector equation (used by the        */
/* learned surrogate; not in the paper).                                     */
/*                                                                           */
/* At steady state the corrector of field j solves (L0 + A) w_j = -v_j with   */
/* L0 = B11 D+D-x + 2 B12 D0x D0y + B22 D+D-y (Fourier symbol -D(k)/h^2,      */
/* D = B11 (2 - 2 cos t1) + B22 (2 - 2 cos t2) + 2 B12 sin t1 sin t2,        */
/* t_i = 2 pi k_i / n) and A w = v1 D0x w + v2 D0y w.  Expanding in v:         */
/*   c_j^0 = -L0^{-1} v_j,  c_j^m = -L0^{-1} A c_j^{m-1},  w_j = sum_m c_j^m,  */
/* so K - B = sum_{m>=2} T_m with T_m = sym <v_i c_j^{m-2}> (mean over the    */
/* cells): T_2 is the small-Peclet limit, T_m is of order v^m.  L0^{-1} is a */
/* division of the DFT by -D/h^2 (the zero mode, where the source has no      */
/* component, set to zero).  The DFT is written out below (separable, plain  */
/* sums); the operators are the patch problem's own (orc_velocity and the    */
/* central differences of Sec. 2.1).                                          */
/* ------------------------------------------------------------------------ */
static void dft2(int n, const double *fr, const double *fi, double *gr, double *gi, int sgn)
{
    double *tr = malloc(sizeof(double) * n * n), *ti = malloc(sizeof(double) * n * n);
    for (int b = 0; b < n; ++b)
        for (int k = 0; k < n; ++k) {
            double sr = 0.0, si = 0.0;
            for (int a = 0; a < n; ++a) {
                double th = sgn * 2.0 * ORC_PI * (double)(((long)k * a) % n) / n;
                double c = cos(th), s = sin(th);
                sr += fr[b * n + a] * c - fi[b * n + a] * s;
                si += fr[b * n + a] * s + fi[b * n + a] * c;
            }
            tr[b * n + k] = sr; ti[b * n + k] = si;
        }
    for (int k2 = 0; k2 < n; ++k2)
        for (int k1 = 0; k1 < n; ++k1) {
            double sr = 0.0, si = 0.0;
            for (int b = 0; b < n; ++b) {
                double th = sgn * 2.0 * ORC_PI * (double)(((long)k2 * b) % n) / n;
                double c = cos(th), s = sin(th);
                sr += tr[b * n + k1] * c - ti[b * n + k1] * s;
                si += tr[b * n + k1] * s + ti[b * n + k1] * c;
            }
            gr[k2 * n + k1] = sr; gi[k2 * n + k1] = si;
        }
    free(tr); free(ti);
}

/* out = -L0^{-1} f for a real field f (mean of f ignored) */
static void neg_l0_inverse(int n, double h, const double *B, const double *f, double *out)
{
    long nn = (long)n * n;
    double *zr = calloc(nn, sizeof(double)), *Fr = malloc(sizeof(double) * nn),
           *Fi = malloc(sizeof(double) * nn), *gi = malloc(sizeof(double) * nn);
    dft2(n, f, zr, Fr, Fi, -1);
    for (int k2 = 0; k2 < n; ++k2)
        for (int k1 = 0; k1 < n; ++k1) {
            long c = (long)k2 * n + k1;
            if (k1 == 0 && k2 == 0) { Fr[c] = Fi[c] = 0.0; continue; }
            double t1 = 2.0 * ORC_PI * k1 / n, t2 = 2.0 * ORC_PI * k2 / n;
            double D = B[0] * (2.0 - 2.0 * cos(t1)) + B[2] * (2.0 - 2.0 * cos(t2))
                     + 2.0 * B[1] * sin(t1) * sin(t2);
            Fr[c] *= h * h / D; Fi[c] *= h * h / D;
        }
    dft2(n, Fr, Fi, out, gi, +1);
    for (long c = 0; c < nn; ++c) out[c] /= (double)nn;
    free(zr); free(Fr); free(Fi); free(gi);
}

/* ------------------------------------------------------------------------ */
/* Periodic-plus-smooth decomposition of a patch field (the periodisation of */
/* a band that is not periodic on the patch; Moisan, "Periodic plus smooth   */
/* image decomposition", 2011).  u = p + s on the n x n samples, where the   */
/* periodic 5-point Laplacian of p equals the Laplacian of u taken over the  */
/* patch's own neighbours only (no neighbour across the seam), and s is the */
/* rest:  Lap_per s = v,  v = Lap_per u - Lap_int u,  which is nonzero on    */
/* the border samples only (v(x) = sum over the seam neighbours y of         */
/* u(y) - u(x)).  s is solved in Fourier space (symbol                       */
/* 2 cos t1 + 2 cos t2 - 4), with mean(s) = 0, so mean(p) = mean(u).         */
/* ------------------------------------------------------------------------ */
void orc_periodic_smooth(int n, const double *u, double *p)
{
    long nn = (long)n * n;
    double *v = calloc(nn, sizeof(double)), *zi = calloc(nn, sizeof(double));
    double *Vr = malloc(sizeof(double) * nn), *Vi = malloc(sizeof(double) * nn);
    double *sr = malloc(sizeof(double) * nn), *si = malloc(sizeof(double) * nn);
    for (int a = 0; a < n; ++a) {          /* rows b = 0 and b = n-1 see each other */
        double j = u[(long)(n - 1) * n + a] - u[a];
        v[a] += j;
        v[(long)(n - 1) * n + a] -= j;
    }
    for (int b = 0; b < n; ++b) {          /* columns a = 0 and a = n-1 */
        double j = u[(long)b * n + n - 1] - u[(long)b * n];
        v[(long)b * n] += j;
        v[(long)b * n + n - 1] -= j;
    }
    dft2(n, v, zi, Vr, Vi, -1);
    for (int k2 = 0; k2 < n; ++k2)
        for (int k1 = 0; k1 < n; ++k1) {
            long c = (long)k2 * n + k1;
            if (k1 == 0 && k2 == 0) { Vr[c] = Vi[c] = 0.0; continue; }
            double d = 2.0 * cos(2.0 * ORC_PI * k1 / n) + 2.0 * cos(2.0 * ORC_PI * k2 / n) - 4.0;
            Vr[c] /= d; Vi[c] /= d;
        }
    dft2(n, Vr, Vi, sr, si, +1);
    for (long c = 0; c < nn; ++c) p[c] = u[c] - sr[c] / (double)nn;
    free(v); free(zi); free(Vr); free(Vi); free(sr); free(si);
}

/* T[(m-2)*3 + (0,1,2)] = (T_m11, T_m12, T_m22) for m = 2..M */
void orc_series(int n, double h, const double *psi, const double *B, int M, double *T)
{
    long nn = (long)n * n;
    double *v1 = malloc(sizeof(double) * nn), *v2 = malloc(sizeof(double) * nn);
    double *c1 = malloc(sizeof(double) * nn), *c2 = malloc(sizeof(double) * nn);
    double *Ac = malloc(sizeof(double) * nn);
    orc_velocity(n, h, psi, v1, v2);
    neg_l0_inverse(n, h, B, v1, c1);
    neg_l0_inverse(n, h, B, v2, c2);
    for (int m = 2; m <= M; ++m) {
        double s11 = 0.0, s12 = 0.0, s21 = 0.0, s22 = 0.0;
        for (long c = 0; c < nn; ++c) {
            s11 += v1[c] * c1[c]; s12 += v1[c] * c2[c];
            s21 += v2[c] * c1[c]; s22 += v2[c] * c2[c];
        }
        T[(m - 2) * 3 + 0] = s11 / nn;
        T[(m - 2) * 3 + 1] = 0.5 * (s12 + s21) / nn;
        T[(m - 2) * 3 + 2] = s22 / nn;
        if (m == M) break;
        for (int j = 0; j < 2; ++j) {
            double *cj = j == 0 ? c1 : c2;
            for (int b = 0; b < n; ++b)
                for (int a = 0; a < n; ++a) {
                    int ap = (a + 1) % n, am = (a + n - 1) % n, bp = (b + 1) % n, bm = (b + n - 1) % n;
                    double dx = (cj[b * n + ap] - cj[b * n + am]) / (2.0 * h);
                    double dy = (cj[bp * n + a] - cj[bm * n + a]) / (2.0 * h);
                    Ac[b * n + a] = v1[b * n + a] * dx + v2[b * n + a] * dy;
                }
            neg_l0_inverse(n, h, B, Ac, cj);
        }
    }
    free(v1); free(v2); free(c1); free(c2); free(Ac);
}

/* Resummation of the series by Wynn's epsilon algorithm (the diagonal Pade   */
/* approximants of a power series at 1): with partial sums S_0..S_{2K},       */
/* eps_{-1}^(j) = 0, eps_0^(j) = S_j,                                          */
/*   eps_{k+1}^(j) = eps_{k-1}^(j+1) + 1 / (eps_k^(j+1) - eps_k^(j)),          */
/* and [K/K] = eps_{2K}^(0).  Where a difference vanishes the last even        */
/* column reached is returned.                                                 */
static double wynn_partial(const double *c, int K)
{
    const int n = 2 * K + 1;
    double *prev = calloc(n + 1, sizeof(double)), *cur = malloc(sizeof(double) * n);
    double *nxt = malloc(sizeof(double) * n);
    double acc = 0.0;
    for (int j = 0; j < n; ++j) { acc += c[j]; cur[j] = acc; }
    double best = cur[n - 1];
    int len = n;
    for (int k = 1; k <= 2 * K; ++k) {
        for (int j = 0; j < len - 1; ++j) {
            double d = cur[j + 1] - cur[j];
            if (fabs(d) < 1e-300) { free(prev); free(cur); free(nxt); return best; }
            nxt[j] = prev[j + 1] + 1.0 / d;
        }
        double *t = prev; prev = cur; cur = nxt; nxt = t;
        len -= 1;
        if (k % 2 == 0) best = cur[0];
    }
    free(prev); free(cur); free(nxt);
    return best;
}

/* [K/K] approximant at x = 1 of the series in x^2 whose terms are the pairs   */
/* p_k = T_(2k+2) + T_(2k+3), k = 0..2K (T_2..T_(4K+3); T: T_2..T_M as          */
/* [M-1][3]), for one component.  K - B is even in v up to the small odd       */
/* moments (the central advection is skew up to O(h^2)), so the pairs are the  */
/* natural terms; an odd moment that vanishes by symmetry then cannot stall   */
/* the epsilon table.                                                          */
double orc_wynn(const double *T, int comp, int K)
{
    double c[32];
    for (int k = 0; k <= 2 * K; ++k) c[k] = T[(2 * k) * 3 + comp] + T[(2 * k + 1) * 3 + comp];
    return wynn_partial(c, K);
}

/* The surrogate's physics estimate of K - B from T_2..T_19: E = [4/4] of the  */
/* pair series, with the lower approximants P2 = [2/2] (T_2..T_11) and         */
/* P3 = [3/3] (T_2..T_15); gap = max_c |E_c - P3_c| measures how far the       */
/* resummation is from converged.                                              */
#define ORC_SERIES_M 19
void orc_series_estimate(const double *T, double *P2, double *P3, double *E, double *gap)
{
    double g = 0.0;
    for (int c = 0; c < 3; ++c) {
        P2[c] = orc_wynn(T, c, 2);
        P3[c] = orc_wynn(T, c, 3);
        E[c] = orc_wynn(T, c, 4);
        double d = fabs(E[c] - P3[c]);
        if (!(d <= g)) g = d;                 /* NaN propagates */
    }
    *gap = g;
}

/* ------------------------------------------------------------------------ */
/* Learned surrogate of the patch solve (not in the paper; the library's     */
/* estimator it is checked against is orc_patch_k).                          */
/*                                                                           */
/* Features of a patch (606 values; a patch above 64 x 64 is described by   */
/* its samples on the 64 x 64 sub-lattice of every (n/64)-th node, with the  */
/* sub-lattice mean removed, and n below stands for 64):                     */
/*   [0, 578): Re and Im of psihat(k) = n^-2 sum_ab psi[b][a]               */
/*             exp(-2 pi i (k1 a + k2 b) / n) for k2 = -8..8 (slow),         */
/*             k1 = -8..8 (fast), each times 32 / (tr(B)/2) (a Peclet        */
/*             scale, brought to order one); psi is the patch's band with    */
/*             the patch mean removed                                        */
/*   578..580: B11/kappa, B12/kappa, B22/kappa;  581: log(kappa)             */
/*   582..596: asinh(10 T_m / tr B) for m = 2..6 (components 11, 12, 22)     */
/*   597..605: asinh(10 x / tr B) for x = P2, P3, E (the [2/2], [3/3], [4/4]  */
/*             approximants of orc_series_estimate)                          */
/*   (the perturbation moments of orc_series and the Wynn approximants of     */
/*   orc_series_estimate; asinh keeps the diverging moments of high-Peclet    */
/*   patches at a usable scale).                                              */
/* Target: asinh((K - B - E) 300 / tr(B)) per component, E = [4/4]; the      */
/* surrogate's K is B + E + tr(B) sinh(out) / 300.                            */
/* ------------------------------------------------------------------------ */
#define ORC_PSI_SCALE 32.0
#define ORC_T_SCALE 10.0
void orc_features(int n, const double *psi, const double *B, double kappa, double *f)
{
    if (n > 64) {
        /* patches above 64 x 64: the features of the samples on the 64 x 64 */
        /* sub-lattice of every (n/64)-th node, sub-lattice mean removed       */
        const int s = n / 64;
        double *q = malloc(sizeof(double) * 64 * 64), mean = 0.0;
        for (int b = 0; b < 64; ++b)
            for (int a = 0; a < 64; ++a) {
                q[b * 64 + a] = psi[(long)(b * s) * n + a * s];
                mean += q[b * 64 + a];
            }
        mean /= 64.0 * 64.0;
        for (int c = 0; c < 64 * 64; ++c) q[c] -= mean;
        orc_features(64, q, B, kappa, f);
        free(q);
        return;
    }
    const double trh = 0.5 * (B[0] + B[2]);
    int t = 0;
    for (int k2 = -8; k2 <= 8; ++k2)
        for (int k1 = -8; k1 <= 8; ++k1) {
            double sr = 0.0, si = 0.0;
            for (int b = 0; b < n; ++b)
                for (int a = 0; a < n; ++a) {
                    long r = pmod((long)k1 * a + (long)k2 * b, n);
                    double th = -2.0 * ORC_PI * (double)r / (double)n;
                    sr += psi[(long)b * n + a] * cos(th);
                    si += psi[(long)b * n + a] * sin(th);
                }
            sr /= (double)n * n;
            si /= (double)n * n;
            f[t++] = sr * ORC_PSI_SCALE / trh;
            f[t++] = si * ORC_PSI_SCALE / trh;
        }
    f[t++] = B[0] / kappa;
    f[t++] = B[1] / kappa;
    f[t++] = B[2] / kappa;
    f[t++] = log(kappa);
    double T[3 * (ORC_SERIES_M - 1)], P2[3], P3[3], E[3], gap;
    orc_series(n, 2.0 * ORC_PI / n, psi, B, ORC_SERIES_M, T);   /* h cancels: any patch side */
    orc_series_estimate(T, P2, P3, E, &gap);
    const double sc = ORC_T_SCALE / (2.0 * trh);
    for (int q = 0; q < 15; ++q) f[t++] = asinh(sc * T[q]);
    for (int c = 0; c < 3; ++c) f[t++] = asinh(sc * P2[c]);
    for (int c = 0; c < 3; ++c) f[t++] = asinh(sc * P3[c]);
    for (int c = 0; c < 3; ++c) f[t++] = asinh(sc * E[c]);
}

/* round to bfloat16 (via float, round to nearest even); NaN-free inputs */
static double bf16r(double x)
{
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    u &= 0xFFFF0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

static double gelu(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }
static double gelu_d(double z)
{
    return 0.5 * (1.0 + erf(z / sqrt(2.0))) + z * exp(-0.5 * z * z) / sqrt(2.0 * ORC_PI);
}

/* One member of the surrogate: 4 dense layers d0 -> h -> h -> h -> 3 with the */
/* exact-erf GELU after the first three.  Parameters (row-major, out x in):    */
/*   W1[h][d0] b1[h] W2[h][h] b2[h] W3[h][h] b3[h] W4[3][h] b4[3]              */
/* in one array.  With bf16 != 0 the inputs, weights and hidden activations    */
/* are rounded to bfloat16 where the GPU stores them in bfloat16, and so are   */
/* the gradients dZ of the hidden layers' pre-activations (the operands of     */
/* the backward contractions); the output layer's dZ stays unrounded.         */
/* Forward: out[M][3].  With Y != NULL also the loss mean((out - Y)^2) over    */
/* the M x 3 entries and its gradient g (same layout as the parameters).       */
double orc_mlp(int M, int d0, int h, const double *X, const double *params, int bf16,
               const double *Y, double *out, double *g)
{
    const int dims[5] = {d0, h, h, h, 3};
    long off[9];
    long o = 0;
    for (int l = 0; l < 4; ++l) { off[2 * l] = o; o += (long)dims[l + 1] * dims[l]; off[2 * l + 1] = o; o += dims[l + 1]; }
    long np = o;
    double *Wq = malloc(sizeof(double) * np);
    for (long q = 0; q < np; ++q) Wq[q] = params[q];
    for (int l = 0; l < 4; ++l)           /* weights in bf16; biases stay FP32 */
        if (bf16) for (long q = off[2 * l]; q < off[2 * l + 1]; ++q) Wq[q] = bf16r(Wq[q]);
    double *A[5], *Z[5];
    for (int l = 0; l <= 4; ++l) { A[l] = malloc(sizeof(double) * M * dims[l]); Z[l] = malloc(sizeof(double) * M * dims[l]); }
    for (long q = 0; q < (long)M * d0; ++q) A[0][q] = bf16 ? bf16r(X[q]) : X[q];
    for (int l = 0; l < 4; ++l) {
        const double *W = Wq + off[2 * l], *bb = Wq + off[2 * l + 1];
        for (int m = 0; m < M; ++m)
            for (int j = 0; j < dims[l + 1]; ++j) {
                double s = bb[j];
                for (int k = 0; k < dims[l]; ++k) s += A[l][(long)m * dims[l] + k] * W[(long)j * dims[l] + k];
                Z[l + 1][(long)m * dims[l + 1] + j] = s;
                double a = (l < 3) ? gelu(s) : s;
                A[l + 1][(long)m * dims[l + 1] + j] = (l < 3 && bf16) ? bf16r(a) : a;
            }
    }
    for (long q = 0; q < (long)M * 3; ++q) out[q] = A[4][q];
    double loss = 0.0;
    if (Y) {
        for (long q = 0; q < (long)M * 3; ++q) loss += (A[4][q] - Y[q]) * (A[4][q] - Y[q]);
        loss /= (double)M * 3.0;
        if (g) {
            /* backward: dZ4 = 2 (out - Y) / (3M); dW = dZ^T A; dA = dZ W; dZ = dA gelu'(Z) */
            double *dZ = malloc(sizeof(double) * M * h), *dA = malloc(sizeof(double) * M * h);
            double *dZn = malloc(sizeof(double) * M * h);
            for (long q = 0; q < (long)M * 3; ++q) dZ[q] = 2.0 * (A[4][q] - Y[q]) / ((double)M * 3.0);
            for (int l = 3; l >= 0; --l) {
                int din = dims[l], dout = dims[l + 1];
                double *gW = g + off[2 * l], *gb = g + off[2 * l + 1];
                const double *W = Wq + off[2 * l];
                for (int j = 0; j < dout; ++j) {
                    double sb = 0.0;
                    for (int m = 0; m < M; ++m) sb += dZ[(long)m * dout + j];
                    gb[j] = sb;
                    for (int k = 0; k < din; ++k) {
                        double s = 0.0;
                        for (int m = 0; m < M; ++m) s += dZ[(long)m * dout + j] * A[l][(long)m * din + k];
                        gW[(long)j * din + k] = s;
                    }
                }
                if (l == 0) break;
                for (int m = 0; m < M; ++m)
                    for (int k = 0; k < din; ++k) {
                        double s = 0.0;
                        for (int j = 0; j < dout; ++j) s += dZ[(long)m * dout + j] * W[(long)j * din + k];
                        const double dz = s * gelu_d(Z[l][(long)m * din + k]);
                        dZn[(long)m * din + k] = bf16 ? bf16r(dz) : dz;
                    }
                double *t = dZ; dZ = dZn; dZn = t;
            }
            free(dZ); free(dA); free(dZn);
        }
    }
    for (int l = 0; l <= 4; ++l) { free(A[l]); free(Z[l]); }
    free(Wq);
    return loss;
}
