// Host runtime and C ABI (include/mlsd.h): level tables, device buffers,
// Algorithm 3 orchestration, error handling.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "mlsd_internal.cuh"

using namespace mlsd;

namespace mlsd {
static std::atomic<long long> g_launches{0};
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace mlsd

namespace {

#define CK(call)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s:%d)",    \
                          #call, cudaGetErrorString(e_), __FILE__, __LINE__);      \
            return e_ == cudaErrorMemoryAllocation ? MLSD_ENOMEM : MLSD_ECUDA;     \
        }                                                                          \
    } while (0)

thread_local char g_last_error[512] = "";

// Patches of one level that share a patch size: one band grid, one kernel.
struct SizeClass {
    int n = 0;
    long long Nl = 0;           // n * m
    double h = 0;
    void *band = nullptr;       // [Nl][Nl] float or double; with periodize: per-patch tiles
    long long tile = 0;         // 0, or n * n: band holds [P][n][n] periodised patch samples
    int *idx = nullptr;         // device patch indices; nullptr when the class holds every patch
    long long count = 0;
    PatchVariant variant{};
    cudaStream_t stream = nullptr;   // own stream when the level has several classes
    cudaEvent_t join = nullptr;
};

struct DevLevel {
    int m = 1;                  // patch side L = 2 pi / m
    double L = 0;
    int n_diag = 0, n_12 = 0, n_21 = 0;
    int nq = 0;                 // largest patch size (stride of the line-variance arrays)
    std::vector<int> np;        // [P] patch size per patch
    int *np_dev = nullptr;      // [P] on the device when sizes are mixed, else nullptr
    double *q12 = nullptr, *q21 = nullptr;   // [P][nq] or null
    double *B = nullptr, *Koff = nullptr, *base = nullptr, *S = nullptr, *Kstar = nullptr;
    long long *steps = nullptr; // [2P] n_burn + n_avg, then n_avg, of the last solve
    std::vector<SizeClass> cls; // largest total work first
    // one launch for every class (patch_level.cu): 0 = per-class launches; 1, 2 = the
    // level kernel with ticket schedule 0 or 1 (largest first, interleaved)
    int lmode = 0;
    long long *tickets[2] = {nullptr, nullptr};
    long long nticket[2] = {0, 0};
    int lv_clusters = 0;        // resident clusters of the level kernel
    cudaEvent_t fork = nullptr;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;   // profiling: one pair per launch
    std::vector<int> ev_n;      // the launch's patch size (0: every class in one launch)
    mlsd_surrogate *sur = nullptr;   // attached surrogate (MLSD_SURROGATE chains) or null
    double sur_thr = 0;
    bool sur_ran = false;            // a surrogate-mode chain ran since the attach
    // workspace of the attached surrogate (sized at attach): series estimates
    // [P][4] FP64, features [P][640] bf16, ensemble outputs [members][P][3],
    // flags [P], compacted fallback indices [P] and their count
    double *sur_E = nullptr;
    void *sur_X = nullptr;
    float *sur_out = nullptr;
    int *sur_flag = nullptr, *sur_idx = nullptr, *sur_cnt = nullptr;
};

}  // namespace

struct mlsd_levels {
    int N = 0;
    long long P = 0;
    int L = 0;
    int precision = MLSD_FP32;
    double kappa = 0, cfl = 0.2, t_burn = 8, t_avg = 4;
    long long nb_fixed = 0, na_fixed = 0;
    std::vector<DevLevel> lev;
    int *status = nullptr;
    std::vector<void *> allocs;
    bool profile = false;
    bool profile_serial = false;     // profiling: a level's size classes one after another
    int n_min = 32, n_max = 256;
    // CUDA graph of the whole Algorithm 3 sequence (captured on first use)
    cudaStream_t cap = nullptr;
    cudaGraphExec_t graph = nullptr;
    const void *graph_out = nullptr, *graph_levels = nullptr;
    long long graph_launches = 0;
    // the same for MLSD_SURROGATE chains (captured again after any attach)
    cudaGraphExec_t graph_sur = nullptr;
    const void *graph_sur_out = nullptr, *graph_sur_levels = nullptr;
    long long graph_sur_launches = 0;
};

namespace {

int dev_alloc(mlsd_levels *h, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) return MLSD_OK;
    CK(cudaMalloc(p, bytes));
    h->allocs.push_back(*p);
    return MLSD_OK;
}

int level_of_mag(int m, int L, const double *e)
{
    for (int l = 1; l <= L; ++l) {
        const double lo = (l == 1) ? 0.0 : e[l - 1];
        if ((double)m >= lo && (double)m < e[l]) return l;
    }
    return L + 1;
}

struct HostMode { int k1, k2; double re, im; };

// group modes by k1 and upload: returns device ModeGroups pointing into `blob`
int upload_groups(mlsd_levels *h, const std::vector<HostMode> &modes, ModeGroups &g)
{
    std::vector<HostMode> ms = modes;
    std::sort(ms.begin(), ms.end(), [](const HostMode &a, const HostMode &b) {
        return a.k1 != b.k1 ? a.k1 < b.k1 : a.k2 < b.k2;
    });
    std::vector<int> gk1, gofs, k2;
    std::vector<double> re, im;
    for (size_t t = 0; t < ms.size(); ++t) {
        if (t == 0 || ms[t].k1 != ms[t - 1].k1) { gk1.push_back(ms[t].k1); gofs.push_back((int)t); }
        k2.push_back(ms[t].k2); re.push_back(ms[t].re); im.push_back(ms[t].im);
    }
    gofs.push_back((int)ms.size());
    g.n_groups = (int)gk1.size();
    if (ms.empty()) { g.gk1 = g.gofs = g.k2 = nullptr; g.re = g.im = nullptr; return MLSD_OK; }
    void *p[5];
    int rc;
    if ((rc = dev_alloc(h, &p[0], gk1.size() * 4))) return rc;
    if ((rc = dev_alloc(h, &p[1], gofs.size() * 4))) return rc;
    if ((rc = dev_alloc(h, &p[2], k2.size() * 4))) return rc;
    if ((rc = dev_alloc(h, &p[3], re.size() * 8))) return rc;
    if ((rc = dev_alloc(h, &p[4], im.size() * 8))) return rc;
    CK(cudaMemcpy(p[0], gk1.data(), gk1.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p[1], gofs.data(), gofs.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p[2], k2.data(), k2.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p[3], re.data(), re.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p[4], im.data(), im.size() * 8, cudaMemcpyHostToDevice));
    g.gk1 = (int *)p[0]; g.gofs = (int *)p[1]; g.k2 = (int *)p[2];
    g.re = (double *)p[3]; g.im = (double *)p[4];
    return MLSD_OK;
}

// refinement of the line samples of Algorithm 1: at least 10 samples per
// wavelength of the finest wavenumber along the line, a multiple of n in all
int line_refine(const std::vector<HostMode> &ms, bool along_x2, double L, int n)
{
    int kmax = 0;
    for (auto &x : ms) kmax = std::max(kmax, std::abs(along_x2 ? x.k2 : x.k1));
    const double need = 10.0 * kmax * L / (2.0 * kPi);
    const int r = (int)std::ceil(need / (double)n);
    return r < 1 ? 1 : r;
}

int validate(const mlsd_problem *p)
{
    if (!p || p->n_macro < 1 || !(p->kappa > 0) || p->n_levels < 1 || p->n_levels > kMaxLevels)
        return MLSD_EINVAL;
    if (p->n_modes < 0 || (p->n_modes > 0 && (!p->k1 || !p->k2 || !p->re || !p->im)))
        return MLSD_EINVAL;
    if (!p->band_edges || !p->patch_n || !(p->cfl > 0)) return MLSD_EINVAL;
    if (p->precision != MLSD_FP32 && p->precision != MLSD_FP64) return MLSD_EINVAL;
    if (p->periodize != 0 && p->periodize != 1) return MLSD_EINVAL;
    for (int l = 0; l < p->n_levels; ++l)
        if (!(p->band_edges[l + 1] > p->band_edges[l])) return MLSD_EINVAL;
    if (p->n_avg_fixed <= 0 && (!(p->t_burn_tau >= 0) || !(p->t_avg_tau > 0))) return MLSD_EINVAL;
    if (p->n_avg_fixed > 0 && p->n_burn_fixed < 0) return MLSD_EINVAL;
    auto pow2in = [](int n) { return n >= 32 && n <= 256 && (n & (n - 1)) == 0; };
    const int nmin = p->n_min ? p->n_min : 32, nmax = p->n_max ? p->n_max : 256;
    if (!pow2in(nmin) || !pow2in(nmax) || nmin > nmax) return MLSD_EINVAL;
    const long long P = (long long)p->n_macro * p->n_macro;
    for (int l = 0; l < p->n_levels; ++l) {
        if (p->patch_n_map) {
            for (long long q = 0; q < P; ++q)
                if (!pow2in(p->patch_n_map[(long long)l * P + q])) return MLSD_EINVAL;
        } else if (p->patch_n[l] != 0 && !pow2in(p->patch_n[l])) {
            return MLSD_EINVAL;
        }
    }
    // Hermitian completeness and no k = 0
    std::map<std::pair<int, int>, std::pair<double, double>> mm;
    for (int t = 0; t < p->n_modes; ++t) {
        if (p->k1[t] == 0 && p->k2[t] == 0) return MLSD_EINVAL;
        if (!std::isfinite(p->re[t]) || !std::isfinite(p->im[t])) return MLSD_EINVAL;
        mm[{p->k1[t], p->k2[t]}] = {p->re[t], p->im[t]};
    }
    for (auto &kv : mm) {
        auto it = mm.find({-kv.first.first, -kv.first.second});
        if (it == mm.end()) return MLSD_EINVAL;
        const double tol = 1e-12 * (std::fabs(kv.second.first) + std::fabs(kv.second.second) + 1e-300);
        if (std::fabs(it->second.first - kv.second.first) > tol ||
            std::fabs(it->second.second + kv.second.second) > tol)
            return MLSD_EINVAL;
    }
    return MLSD_OK;
}

int tune_class(mlsd_levels *h, DevLevel &d, SizeClass &c, cudaStream_t s);
int tune_level(mlsd_levels *h, DevLevel &d, cudaStream_t s);

// Patch size rule for levels given without a size: at least 10 points per
// wavelength of the level's finest diagonal mode and a cell Peclet number of at
// most 2 with kappa (the smallest base any level sees), rounded up to a power of
// two in [n_min, n_max]:  n = pow2ceil(max(10 kmax L / 2pi, L vmax / (2 kappa))).
// vmax is the largest |v| of the band's exact velocity over the patch's
// 32 x 32 reference nodes.
int rule_sizes(mlsd_levels *h, DevLevel &d, const std::vector<HostMode> &diag, cudaStream_t s)
{
    const int nref = 32;
    const long long Nr = (long long)nref * d.m;
    int kmax = 0;
    std::vector<HostMode> c1, c2;            // coefficients of v1 and v2
    for (auto &x : diag) {
        kmax = std::max(kmax, std::max(std::abs(x.k1), std::abs(x.k2)));
        c1.push_back({x.k1, x.k2, x.k2 * x.im, -x.k2 * x.re});
        c2.push_back({x.k1, x.k2, -x.k1 * x.im, x.k1 * x.re});
    }
    std::vector<double> vm((size_t)h->P, 0.0);
    if (!diag.empty()) {
        mlsd_levels tmp;                     // owns the set-up buffers of this step
        ModeGroups g1, g2;
        int rc = upload_groups(&tmp, c1, g1);
        if (!rc) rc = upload_groups(&tmp, c2, g2);
        void *v1 = nullptr, *v2 = nullptr, *G = nullptr, *vmx = nullptr;
        cudaError_t e = cudaSuccess;
        if (!rc) e = cudaMalloc(&v1, (size_t)Nr * Nr * 8);
        if (!rc && e == cudaSuccess) e = cudaMalloc(&v2, (size_t)Nr * Nr * 8);
        if (!rc && e == cudaSuccess) e = cudaMalloc(&G, (size_t)g1.n_groups * Nr * sizeof(double2));
        if (!rc && e == cudaSuccess) e = cudaMalloc(&vmx, (size_t)h->P * 8);
        if (!rc && e == cudaSuccess) e = launch_band_synth(g1, Nr, static_cast<double2 *>(G), v1, 1, s);
        if (!rc && e == cudaSuccess) e = launch_band_synth(g2, Nr, static_cast<double2 *>(G), v2, 1, s);
        if (!rc && e == cudaSuccess)
            e = launch_patch_vmax(static_cast<double *>(v1), static_cast<double *>(v2), Nr, nref,
                                  h->N, h->P, static_cast<double *>(vmx), s);
        if (!rc && e == cudaSuccess) e = cudaMemcpyAsync(vm.data(), vmx, (size_t)h->P * 8, cudaMemcpyDeviceToHost, s);
        if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(s);
        for (void *q : {v1, v2, G, vmx}) if (q) cudaFree(q);
        for (void *q : tmp.allocs) cudaFree(q);
        if (rc) return rc;
        CK(e);
    }
    d.np.resize((size_t)h->P);
    for (long long q = 0; q < h->P; ++q) {
        double need = 10.0 * kmax * d.L / (2.0 * kPi);
        const double pe = d.L * vm[q] / (2.0 * h->kappa);
        if (pe > need) need = pe;
        int n = h->n_min;
        while (n < h->n_max && (double)n < need) n *= 2;
        d.np[q] = n;
    }
    return MLSD_OK;
}

int build(const mlsd_problem *p, cudaStream_t s, mlsd_levels *h)
{
    int rc;
    h->N = p->n_macro;
    h->P = (long long)p->n_macro * p->n_macro;
    h->L = p->n_levels;
    h->precision = p->precision;
    h->kappa = p->kappa;
    h->cfl = p->cfl;
    h->t_burn = p->t_burn_tau;
    h->t_avg = p->t_avg_tau;
    h->nb_fixed = p->n_burn_fixed;
    h->na_fixed = p->n_avg_fixed;
    h->n_min = p->n_min ? p->n_min : 32;
    h->n_max = p->n_max ? p->n_max : 256;
    if ((rc = dev_alloc(h, (void **)&h->status, sizeof(int)))) return rc;
    CK(cudaMemsetAsync(h->status, 0, sizeof(int), s));

    // Sec. 3.1 decomposition: per level, diagonal band and off-diagonal parts
    const int L = p->n_levels;
    std::vector<std::vector<HostMode>> diag(L), off12(L), off21(L);
    for (int t = 0; t < p->n_modes; ++t) {
        const int la = level_of_mag(std::abs(p->k1[t]), L, p->band_edges);
        const int lb = level_of_mag(std::abs(p->k2[t]), L, p->band_edges);
        const HostMode m{p->k1[t], p->k2[t], p->re[t], p->im[t]};
        if (la == lb) { if (la <= L) diag[la - 1].push_back(m); }
        else if (la < lb) off12[la - 1].push_back(m);
        else off21[lb - 1].push_back(m);
    }
    h->lev.resize(L);
    const size_t rs = p->precision == MLSD_FP64 ? 8 : 4;
    for (int l = 0; l < L; ++l) {
        DevLevel &d = h->lev[l];
        if (p->patch_div) d.m = p->patch_div[l];
        else {
            const double e = p->band_edges[l];
            d.m = (int)std::llround(e);
            if (std::fabs(e - d.m) > 0 || d.m < 1) return MLSD_EINVAL;
        }
        if (d.m < 1) return MLSD_EINVAL;
        d.L = 2.0 * kPi / d.m;
        d.n_diag = (int)diag[l].size();
        d.n_12 = (int)off12[l].size();
        d.n_21 = (int)off21[l].size();

        // patch size of every patch: explicit map, one size for the level, or the rule
        if (p->patch_n_map) {
            d.np.assign(p->patch_n_map + (size_t)l * h->P, p->patch_n_map + (size_t)(l + 1) * h->P);
        } else if (p->patch_n[l] > 0) {
            d.np.assign((size_t)h->P, p->patch_n[l]);
        } else if ((rc = rule_sizes(h, d, diag[l], s))) {
            return rc;
        }
        // size classes, largest total work first
        std::map<int, std::vector<int>> by_n;
        for (long long q = 0; q < h->P; ++q) by_n[d.np[q]].push_back((int)q);
        d.nq = by_n.rbegin()->first;
        for (auto it = by_n.rbegin(); it != by_n.rend(); ++it) {
            std::vector<PatchVariant> vs;
            if (patch_variants(it->first, p->precision, vs) == 0) return MLSD_EUNSUPPORTED;
            if (p->periodize && (p->precision != MLSD_FP32 || (it->first != 32 && it->first != 64)))
                return MLSD_EUNSUPPORTED;
            SizeClass c;
            c.n = it->first;
            c.Nl = (long long)c.n * d.m;
            c.h = d.L / c.n;
            c.count = (long long)it->second.size();
            if (by_n.size() > 1) {
                if ((rc = dev_alloc(h, (void **)&c.idx, it->second.size() * sizeof(int)))) return rc;
                CK(cudaMemcpy(c.idx, it->second.data(), it->second.size() * sizeof(int),
                              cudaMemcpyHostToDevice));
            }
            d.cls.push_back(c);
        }
        std::stable_sort(d.cls.begin(), d.cls.end(), [](const SizeClass &a, const SizeClass &b) {
            return (double)a.count * a.n * a.n * a.n > (double)b.count * b.n * b.n * b.n;
        });
        if (d.cls.size() > 1) {
            if ((rc = dev_alloc(h, (void **)&d.np_dev, (size_t)h->P * sizeof(int)))) return rc;
            CK(cudaMemcpy(d.np_dev, d.np.data(), (size_t)h->P * sizeof(int), cudaMemcpyHostToDevice));
            CK(cudaEventCreateWithFlags(&d.fork, cudaEventDisableTiming));
            for (auto &c : d.cls) {
                CK(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
                CK(cudaEventCreateWithFlags(&c.join, cudaEventDisableTiming));
            }
        }

        // band grid of every class (set-up)
        ModeGroups g;
        if ((rc = upload_groups(h, diag[l], g))) return rc;
        for (auto &c : d.cls) {
            if ((rc = dev_alloc(h, &c.band, (size_t)c.Nl * c.Nl * rs))) return rc;
            void *G = nullptr;
            if (g.n_groups > 0) CK(cudaMalloc(&G, (size_t)g.n_groups * c.Nl * sizeof(double2)));
            cudaError_t e = launch_band_synth(g, c.Nl, static_cast<double2 *>(G), c.band,
                                              p->precision == MLSD_FP64, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (G) cudaFree(G);
            CK(e);
            if (p->periodize) {
                // the periodic component of every patch of the class, into its own tile
                void *tiles = nullptr;
                if ((rc = dev_alloc(h, &tiles, (size_t)h->P * c.n * c.n * rs))) return rc;
                CK(launch_periodize(static_cast<const float *>(c.band), c.Nl, c.n, h->N, c.idx,
                                    c.count, static_cast<float *>(tiles), s));
                c.band = tiles;
                c.tile = (long long)c.n * c.n;
            }
        }

        // Algorithm 1 line variances (set-up; independent of the base tensor),
        // factorised: psi_12 grouped by k1 (across its columns), psi_21 by k2
        if (d.n_12 && (rc = dev_alloc(h, (void **)&d.q12, (size_t)h->P * d.nq * 8))) return rc;
        if (d.n_21 && (rc = dev_alloc(h, (void **)&d.q21, (size_t)h->P * d.nq * 8))) return rc;
        if (d.n_12 || d.n_21) {
            mlsd_levels tmp;                 // set-up buffers of this step
            std::vector<HostMode> sw21;
            for (auto &x : off21[l]) sw21.push_back({x.k2, x.k1, x.re, x.im});
            ModeGroups g12, g21;
            rc = upload_groups(&tmp, off12[l], g12);
            if (!rc) rc = upload_groups(&tmp, sw21, g21);
            cudaError_t e = cudaSuccess;
            for (auto &c : d.cls) {
                if (rc || e != cudaSuccess) break;
                const int r12 = line_refine(off12[l], true, d.L, c.n);
                const int r21 = line_refine(off21[l], false, d.L, c.n);
                const size_t need = std::max((size_t)g12.n_groups * c.n * r12,
                                             (size_t)g21.n_groups * c.n * r21) * h->N * sizeof(double2);
                void *G = nullptr;
                e = cudaMalloc(&G, std::max<size_t>(need, 16));
                if (e == cudaSuccess && d.n_12)
                    e = launch_line_var(g12, c.Nl, c.n, r12, h->N, c.count, c.idx, 1, d.nq, d.q12,
                                        static_cast<double2 *>(G), s);
                if (e == cudaSuccess && d.n_21)
                    e = launch_line_var(g21, c.Nl, c.n, r21, h->N, c.count, c.idx, 0, d.nq, d.q21,
                                        static_cast<double2 *>(G), s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (G) cudaFree(G);
            }
            for (void *q : tmp.allocs) cudaFree(q);
            if (rc) return rc;
            CK(e);
        }

        // per-level tensors
        if ((rc = dev_alloc(h, (void **)&d.B, (size_t)h->P * 3 * 8))) return rc;
        if ((rc = dev_alloc(h, (void **)&d.Koff, (size_t)h->P * 3 * 8))) return rc;
        if ((rc = dev_alloc(h, (void **)&d.base, (size_t)h->P * 3 * 8))) return rc;
        if ((rc = dev_alloc(h, (void **)&d.Kstar, (size_t)h->P * 3 * 8))) return rc;
        if ((rc = dev_alloc(h, (void **)&d.S, (size_t)h->P * 4 * 8))) return rc;
        if ((rc = dev_alloc(h, (void **)&d.steps, (size_t)h->P * 16))) return rc;
        CK(cudaMemsetAsync(d.steps, 0, (size_t)h->P * 16, s));
        for (auto &c : d.cls)
            if ((rc = tune_class(h, d, c, s))) return rc;
        if ((rc = tune_level(h, d, s))) return rc;
    }
    CK(cudaStreamSynchronize(s));
    return MLSD_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: time every compiled tiling of the patch kernel on a sample of the
// level's patches (short fixed window, the level's own band, base kappa I) and
// keep the fastest per (device, n, precision) for the rest of the process.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, std::pair<int, int>> g_tune;   // -> (bx, code(by, minb, packed))

int tile_code(const PatchVariant &v)
{
    return v.by * 16 + v.minb + 4096 * v.packed + 65536 * v.cluster + (1 << 24) * v.split +
           (1 << 28) * v.tmem;
}

int tune_class(mlsd_levels *h, DevLevel &d, SizeClass &c, cudaStream_t s)
{
    std::vector<PatchVariant> vs;
    patch_variants(c.n, h->precision, vs);
    if (vs.empty()) return MLSD_EUNSUPPORTED;
    c.variant = vs[0];
    if (const char *env = std::getenv("MLSD_TILE")) {
        // <bx>x<by>[m<minb>][c<cluster>][p][s|n|b|d|r][t|l]: p selects the packed two-field
        // kernel, s the split-phase stage barriers, n neighbour signalling between slabs, b
        // bulk copies of the slab edge rows, d bulk copies with the cross-slab rows computed
        // last, r the row-paired f32x2 kernel, t the per-cell coefficients in tensor memory,
        // l the same with the column halos read as the rows need them
        int bx = 0, by = 0, mb = 1, pk = 0, cl = 1, sp = 0, tm = 0;
        char rest[16] = "";
        if (std::sscanf(env, "%dx%d%15s", &bx, &by, rest) >= 2) {
            for (const char *q = rest; *q; ++q) {
                if (*q == 'm') mb = std::atoi(q + 1);
                if (*q == 'c') cl = std::atoi(q + 1);
                if (*q == 'p') pk = 1;
                if (*q == 's') sp = 1;
                if (*q == 'n') sp = 2;
                if (*q == 'b') sp = 3;
                if (*q == 'r') sp = 4;
                if (*q == 'd') sp = 5;
                if (*q == 't') tm = 1;
                if (*q == 'l') tm = 2;
            }
            for (auto &v : vs)
                if (v.bx == bx && v.by == by && v.minb == mb && v.packed == pk && v.cluster == cl &&
                    v.split == sp && v.tmem == tm) {
                    c.variant = v;
                    return MLSD_OK;
                }
            // the forced tiling is not compiled for this patch size: use the tuner
        } else {
            return MLSD_EINVAL;
        }
    }
    if (vs.size() == 1) return MLSD_OK;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    const auto key = std::make_tuple(dev, c.n, h->precision);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            for (auto &v : vs)
                if (v.bx == it->second.first && tile_code(v) == it->second.second) c.variant = v;
            return MLSD_OK;
        }
    }
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // base kappa I for the sampled patches (the level's B array is free at set-up)
    std::vector<double> kb((size_t)h->P * 3);
    for (long long p = 0; p < h->P; ++p) { kb[3 * p] = h->kappa; kb[3 * p + 1] = 0; kb[3 * p + 2] = h->kappa; }
    CK(cudaMemcpyAsync(d.B, kb.data(), kb.size() * 8, cudaMemcpyHostToDevice, s));
    PatchParams pp;
    pp.band = c.band; pp.Nl = c.Nl; pp.tile = c.tile; pp.n_macro = h->N; pp.h = c.h; pp.L = d.L;
    pp.Kb = d.B; pp.S = d.S; pp.wdump = nullptr; pp.status = h->status;
    // trial window: the problem's own fixed window when it has one (its per-patch
    // set-up share then counts as it will in the solve), else 64 steps, where the
    // stepping rate of a long relaxation window dominates
    pp.cfl = h->cfl; pp.t_burn = 8; pp.t_avg = 4; pp.nb_fixed = 0;
    pp.na_fixed = h->na_fixed > 0 ? std::min<long long>(std::max<long long>(h->nb_fixed + h->na_fixed, 8), 64)
                                  : 64;
    pp.P = h->P; pp.item0 = 0; pp.steps = nullptr; pp.pidx = c.idx;
    pp.items = std::min<long long>(2 * c.count, (long long)sms * (c.n <= 64 ? 48 : 8));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    for (auto &v : vs) {
        float t = 1e30f;
        bool ok = true;
        for (int rep = 0; rep < 3 && ok; ++rep) {
            cudaEventRecord(e0, s);
            ok = launch_patch(v, pp, pp.items, s) == cudaSuccess;
            cudaEventRecord(e1, s);
            if (ok) ok = cudaEventSynchronize(e1) == cudaSuccess;
            float ms = 0.f;
            if (ok && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) t = std::min(t, ms);
        }
        if (!ok) { cudaGetLastError(); continue; }   // a tiling this device cannot launch
        if (std::getenv("MLSD_TUNE_LOG"))
            std::fprintf(stderr, "mlsd tune n=%d items=%lld steps=%lld %dx%d m%d c%d sync%d%s%s: %.4f ms\n",
                         c.n, pp.items, pp.na_fixed, v.bx, v.by, v.minb, v.cluster, v.split,
                         v.packed ? " packed" : "", v.tmem == 2 ? " tmem lazy" : v.tmem ? " tmem" : "", t);
        if (t < best) { best = t; c.variant = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaMemsetAsync(h->status, 0, sizeof(int), s));
    CK(cudaStreamSynchronize(s));
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = {c.variant.bx, tile_code(c.variant)};
    return MLSD_OK;
}

// Size code of a class in the level kernel (LevelParams::cls), or -1: no task shape.
int level_code(int n)
{
    return n == 32 ? 0 : n == 64 ? 1 : n == 128 ? 2 : n == 256 ? 3 : -1;
}

// Ticket list of the level kernel: LevelParams::CLUSTER codes per ticket, each
// (size << 56) | first work item, or -1.  A 256^2 field is one ticket (the
// same code for every CTA of the cluster); the other classes form CTA tasks of
// 65 536 cells (one 128^2, four 64^2 or sixteen 32^2 fields), four per ticket,
// larger patches first.  Schedule 0 puts every 256^2 ticket first; schedule 1
// spreads them evenly among the others.
void build_tickets(const std::vector<std::pair<int, long long>> &classes, int sched,
                   std::vector<long long> &out)
{
    constexpr int CL = LevelParams::CLUSTER;
    std::vector<long long> big, cta;
    for (const auto &c : classes) {
        const int z = level_code(c.first);
        const long long per = z == 1 ? 4 : z == 0 ? 16 : 1;       // fields per task
        for (long long it = 0; it < 2 * c.second; it += per)
            (z == 3 ? big : cta).push_back(((long long)z << 56) | it);
    }
    std::stable_sort(cta.begin(), cta.end(), [](long long a, long long b) { return (a >> 56) > (b >> 56); });
    const long long nb = (long long)big.size(), nq = ((long long)cta.size() + CL - 1) / CL, nt = nb + nq;
    out.clear();
    out.reserve((size_t)(CL * nt));
    long long kb = 0, kq = 0;
    for (long long i = 0; i < nt; ++i) {
        const bool take_big = kb < nb && (kq >= nq || sched == 0 || kb * nt < (i + 1) * nb);
        if (take_big) {
            for (int r = 0; r < CL; ++r) out.push_back(big[kb]);
            ++kb;
        } else {
            for (int r = 0; r < CL; ++r) {
                const long long q = CL * kq + r;
                out.push_back(q < (long long)cta.size() ? cta[q] : -1);
            }
            ++kq;
        }
    }
}

int run_patches(mlsd_levels *h, DevLevel &d, const double *Kb, double *S, void *wdump,
                cudaStream_t s);

// One launch for every class of a mixed-size FP32 level: build both ticket
// schedules and time the whole level (base kappa I, a fixed 16-step window) as
// per-class launches and as the level kernel with either schedule; keep the
// fastest.  MLSD_LEVEL = 0 keeps the per-class launches, 1 or 2 forces the
// level kernel with schedule 0 or 1.
int tune_level(mlsd_levels *h, DevLevel &d, cudaStream_t s)
{
    d.lmode = 0;
    if (h->precision != MLSD_FP32 || d.cls.size() < 2) return MLSD_OK;
    for (const auto &c : d.cls)
        if (level_code(c.n) < 0) return MLSD_OK;
    int force = -1;
    if (const char *env = std::getenv("MLSD_LEVEL")) force = std::atoi(env);
    if (force == 0) return MLSD_OK;
    if (level_kernel_clusters(&d.lv_clusters) != cudaSuccess || d.lv_clusters < 1) {
        cudaGetLastError();
        d.lv_clusters = 0;
        return MLSD_OK;                  // the device cannot hold one cluster of it
    }
    int rc;
    std::vector<std::pair<int, long long>> classes;
    for (const auto &c : d.cls) classes.emplace_back(c.n, c.count);
    for (int k = 0; k < 2; ++k) {
        std::vector<long long> t;
        build_tickets(classes, k, t);
        d.nticket[k] = (long long)t.size() / LevelParams::CLUSTER;
        if ((rc = dev_alloc(h, (void **)&d.tickets[k], t.size() * sizeof(long long)))) return rc;
        CK(cudaMemcpy(d.tickets[k], t.data(), t.size() * sizeof(long long), cudaMemcpyHostToDevice));
    }
    if (force == 1 || force == 2) {
        d.lmode = force;
        return MLSD_OK;
    }
    std::vector<double> kb((size_t)h->P * 3);
    for (long long p = 0; p < h->P; ++p) { kb[3 * p] = h->kappa; kb[3 * p + 1] = 0; kb[3 * p + 2] = h->kappa; }
    CK(cudaMemcpyAsync(d.B, kb.data(), kb.size() * 8, cudaMemcpyHostToDevice, s));
    const long long nb0 = h->nb_fixed, na0 = h->na_fixed;
    const bool prof = h->profile;
    h->nb_fixed = 0;
    h->na_fixed = 16;
    h->profile = false;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    int pick = 0;
    rc = MLSD_OK;
    for (int mode = 0; mode < 3 && !rc; ++mode) {
        d.lmode = mode;
        float t = 1e30f;
        for (int rep = 0; rep < 3 && !rc; ++rep) {
            cudaEventRecord(e0, s);
            rc = run_patches(h, d, d.B, d.S, nullptr, s);
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (!rc && cudaEventSynchronize(e1) == cudaSuccess && rep > 0 &&
                cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
                t = std::min(t, ms);
        }
        if (std::getenv("MLSD_TUNE_LOG"))
            std::fprintf(stderr, "mlsd tune level classes=%d %s: %.4f ms\n", (int)d.cls.size(),
                         mode == 0 ? "per-class launches" : mode == 1 ? "one launch, 256^2 first"
                                                                      : "one launch, interleaved", t);
        if (t < best) { best = t; pick = mode; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->nb_fixed = nb0;
    h->na_fixed = na0;
    h->profile = prof;
    d.lmode = pick;
    if (rc) return rc;
    CK(cudaMemsetAsync(h->status, 0, sizeof(int), s));
    CK(cudaStreamSynchronize(s));
    return MLSD_OK;
}

OffdiagLevel off_of(const DevLevel &d)
{
    OffdiagLevel o;
    o.q12 = d.q12;
    o.q21 = d.q21;
    o.stride = d.nq;
    o.np = d.np_dev;
    return o;
}

PatchParams patch_params(const mlsd_levels *h, const DevLevel &d, const SizeClass &c,
                         const double *Kb, double *S, void *wdump)
{
    PatchParams pp;
    pp.band = c.band;
    pp.Nl = c.Nl;
    pp.tile = c.tile;
    pp.n_macro = h->N;
    pp.h = c.h;
    pp.L = d.L;
    pp.Kb = Kb;
    pp.S = S;
    pp.wdump = wdump;
    pp.status = h->status;
    pp.cfl = h->cfl;
    pp.t_burn = h->t_burn;
    pp.t_avg = h->t_avg;
    pp.nb_fixed = h->nb_fixed;
    pp.na_fixed = h->na_fixed;
    pp.P = h->P;
    pp.item0 = 0;
    pp.items = 2 * c.count;
    pp.steps = d.steps;
    pp.pidx = c.idx;
    return pp;
}

// All patch solves of a level: one launch per size class; with several classes
// they run concurrently on the classes' own streams, forked from and joined to s.
int run_patches(mlsd_levels *h, DevLevel &d, const double *Kb, double *S, void *wdump,
                cudaStream_t s)
{
    if (d.lmode > 0) {
        // every class in one launch of the level kernel
        LevelParams lp{};
        for (const auto &c : d.cls) lp.cls[level_code(c.n)] = patch_params(h, d, c, Kb, S, wdump);
        lp.task = d.tickets[d.lmode - 1];
        lp.n_tickets = d.nticket[d.lmode - 1];
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (h->profile) {
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            CK(cudaEventRecord(e0, s));
        }
        CK(launch_level(lp, d.lv_clusters, s));
        if (h->profile) {
            CK(cudaEventRecord(e1, s));
            d.ev.emplace_back(e0, e1);
            d.ev_n.push_back(0);
        }
        return MLSD_OK;
    }
    const bool fork = d.cls.size() > 1 && !(h->profile && h->profile_serial);
    if (fork) CK(cudaEventRecord(d.fork, s));
    for (auto &c : d.cls) {
        cudaStream_t cs = fork ? c.stream : s;
        if (fork) CK(cudaStreamWaitEvent(cs, d.fork, 0));
        PatchParams pp = patch_params(h, d, c, Kb, S, wdump);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (h->profile) {
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            CK(cudaEventRecord(e0, cs));
        }
        CK(launch_patch(c.variant, pp, pp.items, cs));
        if (h->profile) {
            CK(cudaEventRecord(e1, cs));
            d.ev.emplace_back(e0, e1);
            d.ev_n.push_back(c.n);
        }
        if (fork) {
            CK(cudaEventRecord(c.join, cs));
            CK(cudaStreamWaitEvent(s, c.join, 0));
        }
    }
    return MLSD_OK;
}

void drop_events(DevLevel &d)
{
    for (auto &e : d.ev) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    d.ev.clear();
    d.ev_n.clear();
}

}  // namespace

extern "C" {

const char *mlsd_strerror(int code)
{
    switch (code) {
    case MLSD_OK: return "ok";
    case MLSD_EINVAL: return "invalid argument";
    case MLSD_ENOMEM: return "out of memory";
    case MLSD_ECUDA: return g_last_error[0] ? g_last_error : "CUDA error";
    case MLSD_ETIMEOUT: return "device wait timed out";
    case MLSD_ENONFINITE: return "non-finite value in a result";
    case MLSD_EUNSUPPORTED: return "unsupported configuration";
    default: return "unknown error";
    }
}

int mlsd_build_levels(const mlsd_problem *p, void *cuda_stream, mlsd_levels **out)
{
    if (!out) return MLSD_EINVAL;
    *out = nullptr;
    int rc = validate(p);
    if (rc) return rc;
    mlsd_levels *h = new (std::nothrow) mlsd_levels();
    if (!h) return MLSD_ENOMEM;
    rc = build(p, static_cast<cudaStream_t>(cuda_stream), h);
    if (rc) { mlsd_free_levels(h); return rc; }
    *out = h;
    return MLSD_OK;
}

void mlsd_free_levels(mlsd_levels *h)
{
    if (!h) return;
    cudaDeviceSynchronize();
    for (auto &d : h->lev) {
        drop_events(d);
        for (auto &c : d.cls) {
            if (c.stream) cudaStreamDestroy(c.stream);
            if (c.join) cudaEventDestroy(c.join);
        }
        if (d.fork) cudaEventDestroy(d.fork);
    }
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->graph_sur) cudaGraphExecDestroy(h->graph_sur);
    if (h->cap) cudaStreamDestroy(h->cap);
    for (void *p : h->allocs) cudaFree(p);
    delete h;
}

int mlsd_level_info(const mlsd_levels *h, int level, mlsd_level_desc *out)
{
    if (!h || !out || level < 1 || level > h->L) return MLSD_EINVAL;
    const DevLevel &d = h->lev[level - 1];
    const SizeClass &c = d.cls[0];
    out->n = c.n;
    out->Nl = c.Nl;
    out->L = d.L;
    out->h = c.h;
    out->n_patches = h->P;
    out->n_diag_modes = d.n_diag;
    out->n_off12_modes = d.n_12;
    out->n_off21_modes = d.n_21;
    out->tile_bx = c.variant.bx;
    out->tile_by = c.variant.by;
    out->threads = c.variant.threads;
    out->packed = c.variant.packed;
    out->cluster = c.variant.cluster;
    out->min_ctas = c.variant.minb;
    out->split = c.variant.split;
    out->n_classes = (int)d.cls.size();
    out->coef_tmem = c.variant.tmem;
    out->level_launch = d.lmode;
    return MLSD_OK;
}

int mlsd_patch_sizes(const mlsd_levels *h, int level, int32_t *n_out_host)
{
    if (!h || !n_out_host || level < 1 || level > h->L) return MLSD_EINVAL;
    const DevLevel &d = h->lev[level - 1];
    std::copy(d.np.begin(), d.np.end(), n_out_host);
    return MLSD_OK;
}

int mlsd_solve_level(mlsd_levels *h, int level, const double *K_base_dev, double *K_out_dev,
                     void *w_dump_dev, void *cuda_stream)
{
    if (!h || level < 1 || level > h->L || !K_base_dev || !K_out_dev || K_base_dev == K_out_dev)
        return MLSD_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    DevLevel &d = h->lev[level - 1];
    if (w_dump_dev && d.cls.size() > 1) return MLSD_EINVAL;   // dump layout needs one patch size
    int rc = run_patches(h, d, K_base_dev, d.S, w_dump_dev, s);
    if (rc) return rc;
    CK(launch_compose(h->P, K_base_dev, d.S, K_out_dev, h->status, s));
    return MLSD_OK;
}

int mlsd_offdiag(mlsd_levels *h, int level, const double *B_dev, double *Koff_dev,
                 void *cuda_stream)
{
    if (!h || level < 1 || level > h->L || !B_dev || !Koff_dev) return MLSD_EINVAL;
    CK(launch_offdiag_apply(h->P, off_of(h->lev[level - 1]), B_dev, Koff_dev,
                            static_cast<cudaStream_t>(cuda_stream)));
    return MLSD_OK;
}

}  // extern "C"

namespace {
int surrogate_level_async(mlsd_levels *h, DevLevel &d, cudaStream_t s);
// patch sizes the surrogate's features serve (above 64: on the 64 x 64 sub-lattice)
inline bool sur_size_ok(int n) { return n == 32 || n == 64 || n == 128 || n == 256; }
int surrogate_workspace(mlsd_levels *h, DevLevel &d, mlsd_surrogate *sur);

// Algorithm 3 over all levels, enqueued on stream s
int enqueue_chain(mlsd_levels *h, double *K_macro_dev, double *K_levels_dev, cudaStream_t s,
                  bool surrogate = false)
{
    const int L = h->L;
    ChainTables t;
    t.L = L;
    t.P = h->P;
    t.kappa = h->kappa;
    for (int l = 0; l < L; ++l) {
        t.off[l] = off_of(h->lev[l]);
        t.B[l] = h->lev[l].B;
        t.Koff[l] = h->lev[l].Koff;
    }
    CK(launch_topdown(t, s));
    for (int l = L - 1; l >= 0; --l) {
        DevLevel &d = h->lev[l];
        const bool finest = (l == L - 1);
        const DevLevel *nx = finest ? nullptr : &h->lev[l + 1];
        CK(launch_level_base(h->P, finest ? 1 : 0, nx ? nx->base : nullptr, nx ? nx->S : nullptr,
                             nx ? nx->Kstar : nullptr, d.Koff, d.B, off_of(d), d.base, s));
        int rc;
        if (surrogate && d.sur) {
            // the level's K* from the ensemble (plain solves where it is unsure), then
            // S = K* - base so that the rest of the chain reads it like a plain solve;
            // the step counts then cover the fallback solves only.  No host
            // synchronisation: the fallback launch reads its count on the device.
            CK(cudaMemsetAsync(d.steps, 0, (size_t)h->P * 16, s));
            rc = surrogate_level_async(h, d, s);
            if (!rc) CK(launch_S_from_K(h->P, d.base, d.Kstar, d.S, s));
        } else {
            rc = run_patches(h, d, d.base, d.S, nullptr, s);
        }
        if (rc) return rc;
    }
    DevLevel &c = h->lev[0];
    CK(launch_compose(h->P, c.base, c.S, c.Kstar, h->status, s));
    CK(cudaMemcpyAsync(K_macro_dev, c.Kstar, (size_t)h->P * 3 * 8, cudaMemcpyDeviceToDevice, s));
    if (K_levels_dev) {
        for (int l = 0; l < L; ++l)
            CK(cudaMemcpyAsync(K_levels_dev + (size_t)l * h->P * 3, h->lev[l].Kstar,
                               (size_t)h->P * 3 * 8, cudaMemcpyDeviceToDevice, s));
    }
    return MLSD_OK;
}
}  // namespace

extern "C" {

int mlsd_effective_diffusivity(mlsd_levels *h, int mode, double *K_macro_dev,
                               double *K_levels_dev, void *cuda_stream)
{
    if (!h || !K_macro_dev || (mode != MLSD_PLAIN && mode != MLSD_SURROGATE)) return MLSD_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (mode == MLSD_SURROGATE) {
        bool any = false;
        for (DevLevel &d : h->lev) any = any || d.sur;
        if (!any) return MLSD_EINVAL;
        for (DevLevel &d : h->lev) d.sur_ran = d.sur != nullptr;
        if (h->profile || std::getenv("MLSD_NO_GRAPH"))
            return enqueue_chain(h, K_macro_dev, K_levels_dev, s, true);
        if (!h->graph_sur || h->graph_sur_out != K_macro_dev || h->graph_sur_levels != K_levels_dev) {
            if (h->graph_sur) { cudaGraphExecDestroy(h->graph_sur); h->graph_sur = nullptr; }
            if (!h->cap) CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
            const long long n0 = launch_count();
            CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
            int rc = enqueue_chain(h, K_macro_dev, K_levels_dev, h->cap, true);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(h->cap, &g);
            if (rc) { if (g) cudaGraphDestroy(g); return rc; }
            CK(e);
            e = cudaGraphInstantiate(&h->graph_sur, g, 0);
            cudaGraphDestroy(g);
            CK(e);
            h->graph_sur_out = K_macro_dev;
            h->graph_sur_levels = K_levels_dev;
            h->graph_sur_launches = launch_count() - n0;
            count_launches(-h->graph_sur_launches);
        }
        CK(cudaGraphLaunch(h->graph_sur, s));
        count_launches(h->graph_sur_launches);
        return MLSD_OK;
    }
    // profiling records events per launch: run the sequence directly then
    if (h->profile || std::getenv("MLSD_NO_GRAPH")) return enqueue_chain(h, K_macro_dev, K_levels_dev, s);
    if (!h->graph || h->graph_out != K_macro_dev || h->graph_levels != K_levels_dev) {
        if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
        if (!h->cap) CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
        const long long n0 = launch_count();
        CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_chain(h, K_macro_dev, K_levels_dev, h->cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->cap, &g);
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        CK(e);
        e = cudaGraphInstantiate(&h->graph, g, 0);
        cudaGraphDestroy(g);
        CK(e);
        h->graph_out = K_macro_dev;
        h->graph_levels = K_levels_dev;
        h->graph_launches = launch_count() - n0;
        count_launches(-h->graph_launches);      // capture launched nothing
    }
    CK(cudaGraphLaunch(h->graph, s));
    count_launches(h->graph_launches);
    return MLSD_OK;
}

int mlsd_attach_surrogate(mlsd_levels *h, int level, mlsd_surrogate *s, double threshold)
{
    if (!h || level < 1 || level > h->L || !(threshold >= 0)) return MLSD_EINVAL;
    DevLevel &d = h->lev[level - 1];
    if (s && (d.cls.size() != 1 || !sur_size_ok(d.cls[0].n) ||
              h->precision != MLSD_FP32))
        return MLSD_EUNSUPPORTED;
    if (s) {
        int rc = surrogate_workspace(h, d, s);
        if (rc) return rc;
    }
    d.sur = s;
    d.sur_thr = threshold;
    d.sur_ran = false;
    if (h->graph_sur) { cudaGraphExecDestroy(h->graph_sur); h->graph_sur = nullptr; }
    return MLSD_OK;
}

int mlsd_surrogate_fallbacks(mlsd_levels *h, int level, int64_t *n_out)
{
    if (!h || level < 1 || level > h->L || !n_out) return MLSD_EINVAL;
    const DevLevel &d = h->lev[level - 1];
    *n_out = -1;
    if (!d.sur || !d.sur_ran || !d.sur_cnt) return MLSD_OK;
    int n = 0;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(&n, d.sur_cnt, sizeof(int), cudaMemcpyDeviceToHost));
    *n_out = n;
    return MLSD_OK;
}

int mlsd_status(mlsd_levels *h, void *cuda_stream)
{
    if (!h) return MLSD_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    CK(cudaStreamSynchronize(s));
    int v = 0;
    CK(cudaMemcpy(&v, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (v) CK(cudaMemset(h->status, 0, sizeof(int)));
    return v;
}

int mlsd_check_wait_timeout(mlsd_levels *h, int which, void *cuda_stream)
{
    if (!h || which < 0 || which > 2) return MLSD_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    CK(which == 0 ? launch_wait_check_nbr(h->status, s)
       : which == 1 ? launch_wait_check_mbar(h->status, s) : launch_wait_check_tile(h->status, s));
    return MLSD_OK;
}

int mlsd_corrector_energy(mlsd_levels *h, int level, const double *K_base_dev, const void *w_dump_dev,
                          double *E_out_dev, double *mass_out_dev, void *cuda_stream)
{
    if (!h || level < 1 || level > h->L || !K_base_dev || !w_dump_dev || !E_out_dev) return MLSD_EINVAL;
    const DevLevel &d = h->lev[level - 1];
    if (d.cls.size() != 1) return MLSD_EINVAL;                  // the dump layout needs one size
    const SizeClass &c = d.cls[0];
    CK(launch_corrector_energy(c.n, c.h, h->P, h->precision, w_dump_dev, K_base_dev, E_out_dev,
                               mass_out_dev, static_cast<cudaStream_t>(cuda_stream)));
    return MLSD_OK;
}

int mlsd_level_work(mlsd_levels *h, int level, int64_t *cell_updates_out,
                    int64_t *window_updates_out, int64_t *max_steps_out, void *cuda_stream)
{
    if (!h || level < 1 || level > h->L) return MLSD_EINVAL;
    const DevLevel &d = h->lev[level - 1];
    std::vector<long long> st((size_t)h->P * 2);
    CK(cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream)));
    CK(cudaMemcpy(st.data(), d.steps, (size_t)h->P * 16, cudaMemcpyDeviceToHost));
    long long tot = 0, win = 0, mx = 0;
    for (long long q = 0; q < h->P; ++q) {
        const long long cells = 2 * (long long)d.np[q] * d.np[q];
        tot += st[q] * cells;
        win += st[h->P + q] * cells;
        mx = std::max(mx, st[q]);
    }
    if (cell_updates_out) *cell_updates_out = tot;
    if (window_updates_out) *window_updates_out = win;
    if (max_steps_out) *max_steps_out = mx;
    return MLSD_OK;
}

int64_t mlsd_launch_count(void) { return launch_count(); }

int mlsd_level_schedule(const int32_t *patch_n, const int64_t *patches, int n_classes, int schedule,
                        int64_t capacity, int64_t *codes_out, int64_t *n_tickets_out)
{
    if (!patch_n || !patches || n_classes < 1 || n_classes > 4 || schedule < 0 || schedule > 1 ||
        capacity < 0 || !n_tickets_out || (capacity > 0 && !codes_out))
        return MLSD_EINVAL;
    std::vector<std::pair<int, long long>> classes;
    for (int i = 0; i < n_classes; ++i) {
        if (level_code(patch_n[i]) < 0 || patches[i] < 1) return MLSD_EINVAL;
        for (const auto &c : classes)
            if (c.first == patch_n[i]) return MLSD_EINVAL;
        classes.emplace_back(patch_n[i], (long long)patches[i]);
    }
    std::vector<long long> t;
    build_tickets(classes, schedule, t);
    *n_tickets_out = (int64_t)t.size() / LevelParams::CLUSTER;
    if ((int64_t)t.size() > capacity) return MLSD_EINVAL;
    std::copy(t.begin(), t.end(), codes_out);
    return MLSD_OK;
}

int mlsd_profile(mlsd_levels *h, int enable)
{
    if (!h || enable < 0 || enable > 2) return MLSD_EINVAL;
    h->profile = enable != 0;
    h->profile_serial = enable == 2;
    return MLSD_OK;
}

int mlsd_profile_collect_classes(mlsd_levels *h, int level, int capacity, int32_t *patch_n_out,
                                 double *kernel_ms_out, int64_t *launches_out, int32_t *n_written)
{
    if (!h || level < 1 || level > h->L || capacity < 0 || !n_written ||
        (capacity > 0 && (!patch_n_out || !kernel_ms_out || !launches_out)))
        return MLSD_EINVAL;
    DevLevel &d = h->lev[level - 1];
    std::vector<int> ns;
    std::vector<double> ms;
    std::vector<int64_t> cnt;
    for (size_t i = 0; i < d.ev.size(); ++i) {
        CK(cudaEventSynchronize(d.ev[i].second));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, d.ev[i].first, d.ev[i].second));
        const int n = d.ev_n[i];
        size_t k = 0;
        while (k < ns.size() && ns[k] != n) ++k;
        if (k == ns.size()) { ns.push_back(n); ms.push_back(0.0); cnt.push_back(0); }
        ms[k] += t;
        cnt[k] += 1;
    }
    if ((int)ns.size() > capacity) return MLSD_EINVAL;   // events kept for a larger call
    for (size_t k = 0; k < ns.size(); ++k) {
        patch_n_out[k] = ns[k];
        kernel_ms_out[k] = ms[k];
        launches_out[k] = cnt[k];
    }
    *n_written = (int32_t)ns.size();
    drop_events(d);
    return MLSD_OK;
}

int mlsd_profile_collect(mlsd_levels *h, int level, double *kernel_ms_out, int64_t *launches_out)
{
    if (!h || level < 1 || level > h->L) return MLSD_EINVAL;
    DevLevel &d = h->lev[level - 1];
    double tot = 0.0;
    for (auto &e : d.ev) {
        CK(cudaEventSynchronize(e.second));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e.first, e.second));
        tot += ms;
    }
    if (kernel_ms_out) *kernel_ms_out = tot;
    if (launches_out) *launches_out = (int64_t)d.ev.size();
    drop_events(d);
    return MLSD_OK;
}

int mlsd_macro_step(int n_macro, void *U_dev, int precision, const double *K_dev, double dt,
                    int nsteps, double *mass_out_host, void *cuda_stream)
{
    if (n_macro < 2 || !U_dev || !K_dev || !(dt > 0) || nsteps < 0) return MLSD_EINVAL;
    if (precision != MLSD_FP32 && precision != MLSD_FP64) return MLSD_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const size_t sb = macro_scratch_bytes(n_macro, precision, nsteps);
    const size_t mb = mass_out_host ? (size_t)(nsteps + 1) * sizeof(double) : 0;
    void *scratch = nullptr;
    if (sb + mb) CK(cudaMallocAsync(&scratch, sb + mb + 256, s));
    double *mass = mass_out_host
        ? reinterpret_cast<double *>((reinterpret_cast<uintptr_t>(scratch) + sb + 255) & ~(uintptr_t)255)
        : nullptr;
    cudaError_t e = macro_run(n_macro, U_dev, precision, K_dev, dt, nsteps, mass, scratch, s);
    if (e == cudaSuccess && mass_out_host)
        e = cudaMemcpyAsync(mass_out_host, mass, mb, cudaMemcpyDeviceToHost, s);
    if (scratch) cudaFreeAsync(scratch, s);
    if (e == cudaSuccess && mass_out_host) e = cudaStreamSynchronize(s);
    CK(e);
    return MLSD_OK;
}

int mlsd_macro_step_dirichlet(int n_macro, void *U_dev, int precision, const double *K_dev,
                              double dt, int nsteps, double u_left, double u_right,
                              double *mass_out_host, void *cuda_stream)
{
    if (n_macro < 2 || !U_dev || !K_dev || !(dt > 0) || nsteps < 0) return MLSD_EINVAL;
    if (precision != MLSD_FP32 && precision != MLSD_FP64) return MLSD_EINVAL;
    if (!std::isfinite(u_left) || !std::isfinite(u_right)) return MLSD_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const size_t sb = macro_scratch_bytes(n_macro, precision, nsteps);
    const size_t mb = mass_out_host ? (size_t)(nsteps + 1) * sizeof(double) : 0;
    void *scratch = nullptr;
    if (sb + mb) CK(cudaMallocAsync(&scratch, sb + mb + 256, s));
    double *mass = mass_out_host
        ? reinterpret_cast<double *>((reinterpret_cast<uintptr_t>(scratch) + sb + 255) & ~(uintptr_t)255)
        : nullptr;
    cudaError_t e = macro_run_dirichlet(n_macro, U_dev, precision, K_dev, dt, nsteps, u_left,
                                        u_right, mass, scratch, s);
    if (e == cudaSuccess && mass_out_host)
        e = cudaMemcpyAsync(mass_out_host, mass, mb, cudaMemcpyDeviceToHost, s);
    if (scratch) cudaFreeAsync(scratch, s);
    if (e == cudaSuccess && mass_out_host) e = cudaStreamSynchronize(s);
    CK(e);
    return MLSD_OK;
}

int mlsd_macro_dt(int n_macro, const double *K_dev, double cfl, double *dt_out_host,
                  void *cuda_stream)
{
    if (n_macro < 2 || !K_dev || !(cfl > 0) || !dt_out_host) return MLSD_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    double *m = nullptr;
    CK(cudaMallocAsync((void **)&m, sizeof(double), s));
    cudaError_t e = macro_dt_max(n_macro, K_dev, m, s);
    double mx = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&mx, m, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(m, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    CK(e);
    if (!(mx > 0) || !std::isfinite(mx)) return MLSD_ENONFINITE;
    const double H = 2.0 * kPi / n_macro;
    *dt_out_host = cfl * H * H / mx;
    return MLSD_OK;
}

int mlsd_grid_psi(int n_modes, const int32_t *k1, const int32_t *k2, const double *re,
                  const double *im, int nf, float *psi_dev, void *cuda_stream)
{
    if (n_modes < 0 || nf < 1 || !psi_dev || (n_modes > 0 && (!k1 || !k2 || !re || !im)))
        return MLSD_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    mlsd_levels tmp;   // owns the staging buffers for this call only
    std::vector<HostMode> ms;
    for (int t = 0; t < n_modes; ++t) ms.push_back({k1[t], k2[t], re[t], im[t]});
    ModeGroups g;
    int rc = upload_groups(&tmp, ms, g);
    void *G = nullptr;
    cudaError_t e = cudaSuccess;
    if (!rc && g.n_groups > 0) e = cudaMalloc(&G, (size_t)g.n_groups * nf * sizeof(double2));
    if (!rc && e == cudaSuccess) e = launch_band_synth(g, nf, static_cast<double2 *>(G), psi_dev, 0, s);
    if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (G) cudaFree(G);
    for (void *p : tmp.allocs) cudaFree(p);
    if (rc) return rc;
    CK(e);
    return MLSD_OK;
}

int mlsd_dns_run(int nf, float *u_dev, float *u_tmp_dev, const float *psi_dev, double kappa,
                 double dt, int nsteps, void *cuda_stream)
{
    if (nf < 128 || nf % 128 || !u_dev || !u_tmp_dev || !psi_dev || u_dev == u_tmp_dev ||
        !(kappa >= 0) || !(dt > 0) || nsteps < 0)
        return MLSD_EINVAL;
    CK(dns_run(nf, u_dev, u_tmp_dev, psi_dev, kappa, dt, nsteps,
               static_cast<cudaStream_t>(cuda_stream)));
    return MLSD_OK;
}

int mlsd_dns_status(void *cuda_stream)
{
    return dns_status_take(static_cast<cudaStream_t>(cuda_stream));
}

const char *mlsd_dns_kernel(void)
{
    return dns_kernel_name();
}

int mlsd_dns_run_dirichlet(int nf, void *u_dev, void *u_tmp_dev, const float *psi_dev,
                           int precision, double kappa, double dt, int nsteps, double u_left,
                           double u_right, void *cuda_stream)
{
    if (nf < 4 || !u_dev || !u_tmp_dev || !psi_dev || u_dev == u_tmp_dev || !(kappa >= 0) ||
        !(dt > 0) || nsteps < 0 || !std::isfinite(u_left) || !std::isfinite(u_right))
        return MLSD_EINVAL;
    if (precision != MLSD_FP32 && precision != MLSD_FP64) return MLSD_EINVAL;
    CK(dns_run_dirichlet(nf, u_dev, u_tmp_dev, psi_dev, precision, kappa, dt, nsteps, u_left,
                         u_right, static_cast<cudaStream_t>(cuda_stream)));
    return MLSD_OK;
}

int mlsd_dns_dt(int nf, const float *psi_dev, double kappa, double cfl, double *dt_out_host,
                void *cuda_stream)
{
    if (nf < 2 || !psi_dev || !(kappa > 0) || !(cfl > 0) || !dt_out_host) return MLSD_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    unsigned *m = nullptr;
    CK(cudaMallocAsync((void **)&m, sizeof(unsigned), s));
    cudaError_t e = dns_vmax(nf, psi_dev, m, s);
    unsigned bits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, m, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(m, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    CK(e);
    float vmax;
    std::memcpy(&vmax, &bits, sizeof(float));
    if (!std::isfinite(vmax)) return MLSD_ENONFINITE;
    const double h = 2.0 * kPi / nf;
    double dt = h * h / (4.0 * kappa);
    if (vmax > 0) dt = std::min(dt, h / (double)vmax);
    *dt_out_host = cfl * dt;
    return MLSD_OK;
}

int mlsd_coarse_grain(int nf, const float *u_dev, int n_macro, float *U_dev,
                      double *mass_out_host, void *cuda_stream)
{
    if (nf < 1 || n_macro < 1 || nf % n_macro || !u_dev || !U_dev) return MLSD_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    double *m = nullptr;
    if (mass_out_host)
        CK(cudaMallocAsync((void **)&m, (1 + (size_t)n_macro * n_macro) * sizeof(double), s));
    cudaError_t e = coarse_grain(nf, u_dev, n_macro, U_dev, m, s);
    if (e == cudaSuccess && m) e = cudaMemcpyAsync(mass_out_host, m, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (m) cudaFreeAsync(m, s);
    if (e == cudaSuccess && m) e = cudaStreamSynchronize(s);
    CK(e);
    return MLSD_OK;
}


}  // extern "C"

// ---------------------------------------------------------------------------
// Surrogate handle
struct mlsd_surrogate {
    int members = 0, h = 0, max_batch = 0;
    long long np = 0;
    std::vector<float *> w, g, m, v;      // FP32 master, gradient, Adam moments
    std::vector<void *> wb;               // bfloat16 copies
    std::vector<int> t;                   // Adam step per member
    float *Z[4] = {};
    void *A[3] = {};
    float *dA = nullptr, *dB = nullptr;
    float *ws = nullptr;                  // split-k partials of the training GEMMs
    long long ws_n = 0;
    double *part = nullptr, *loss = nullptr;
    void **wb_ptrs = nullptr;             // device arrays of the members' parameter pointers
    float **wf_ptrs = nullptr;
    int *status = nullptr;
    int engine = MLSD_SUR_CUDA;
    bool tma = false;                     // TMA-fed tensor-core kernel available
    std::vector<unsigned char> maps;      // its weight tensor maps
    bool train_tc = false;                // training contractions on the tensor cores
    SurTc tc;                             // their buffers
    std::vector<void *> allocs;
};

namespace {
int sur_alloc(mlsd_surrogate *s, void **p, size_t bytes)
{
    *p = nullptr;
    CK(cudaMalloc(p, bytes));
    s->allocs.push_back(*p);
    return MLSD_OK;
}

// gradient of one member on M rows: the hidden layers' contractions on the tensor
// cores when the handle has their buffers, else every GEMM on the CUDA cores
cudaError_t grad_of(mlsd_surrogate *s, int member, int M, const void *X, const float *Y, float *g,
                    double *part, double *loss, float *ws, long long ws_n, cudaStream_t st)
{
    if (s->train_tc && M <= s->tc.max_rows)
        return sur_grad_tc(s->h, M, X, Y, s->w[member], s->wb[member], s->Z, s->A, s->dA, s->dB,
                           g, part, loss, ws, ws_n, s->tc, s->status, st);
    return sur_grad(s->h, M, X, Y, s->w[member], s->wb[member], s->Z, s->A, s->dA, s->dB, g, part,
                    loss, ws, ws_n, st);
}
}  // namespace

extern "C" {

int64_t mlsd_surrogate_param_count(int hidden) { return sur_param_count(hidden); }

void mlsd_surrogate_free(mlsd_surrogate *s)
{
    if (!s) return;
    cudaDeviceSynchronize();
    for (void *p : s->allocs) cudaFree(p);
    delete s;
}

int mlsd_surrogate_create(int members, int hidden, int max_batch, mlsd_surrogate **out)
{
    if (!out || members < 1 || members > 16 || hidden < 32 || hidden > 512 || hidden % 32 ||
        max_batch < 1)
        return MLSD_EINVAL;
    *out = nullptr;
    mlsd_surrogate *s = new (std::nothrow) mlsd_surrogate();
    if (!s) return MLSD_ENOMEM;
    s->members = members;
    s->h = hidden;
    s->max_batch = max_batch;
    s->np = sur_param_count(hidden);
    int rc = MLSD_OK;
    const size_t np = (size_t)s->np, M = (size_t)max_batch, H = (size_t)hidden;
    for (int k = 0; k < members && !rc; ++k) {
        void *p[5];
        for (int q = 0; q < 4 && !rc; ++q) rc = sur_alloc(s, &p[q], np * 4);
        if (!rc) rc = sur_alloc(s, &p[4], np * 2);
        if (rc) break;
        s->w.push_back((float *)p[0]); s->g.push_back((float *)p[1]);
        s->m.push_back((float *)p[2]); s->v.push_back((float *)p[3]);
        s->wb.push_back(p[4]);
        s->t.push_back(0);
        for (int q = 0; q < 5; ++q) if (cudaMemset(p[q], 0, q < 4 ? np * 4 : np * 2)) rc = MLSD_ECUDA;
    }
    for (int l = 0; l < 4 && !rc; ++l) rc = sur_alloc(s, (void **)&s->Z[l], M * (l < 3 ? H : 3) * 4);
    for (int l = 0; l < 3 && !rc; ++l) rc = sur_alloc(s, &s->A[l], M * H * 2);
    if (!rc) rc = sur_alloc(s, (void **)&s->dA, M * H * 4);
    if (!rc) rc = sur_alloc(s, (void **)&s->dB, M * H * 4);
    s->ws_n = sur_split_workspace(hidden);
    if (!rc) rc = sur_alloc(s, (void **)&s->ws, (size_t)s->ws_n * 4);
    if (!rc) rc = sur_alloc(s, (void **)&s->part, ((3 * M + 255) / 256 + 1) * 8);
    if (!rc) rc = sur_alloc(s, (void **)&s->loss, 8);
    if (!rc) rc = sur_alloc(s, (void **)&s->wb_ptrs, members * sizeof(void *));
    if (!rc) rc = sur_alloc(s, (void **)&s->wf_ptrs, members * sizeof(float *));
    if (!rc) rc = sur_alloc(s, (void **)&s->status, sizeof(int));
    if (!rc) {
        if (cudaMemcpy(s->wb_ptrs, s->wb.data(), members * sizeof(void *), cudaMemcpyHostToDevice) ||
            cudaMemcpy(s->wf_ptrs, s->w.data(), members * sizeof(float *), cudaMemcpyHostToDevice) ||
            cudaMemset(s->status, 0, sizeof(int)))
            rc = MLSD_ECUDA;
    }
    if (!rc && mlp_tc_supported(hidden)) s->engine = MLSD_SUR_TENSOR;
    if (!rc && !std::getenv("MLSD_NO_TMA")) {
        s->maps.assign(mlp_tma_maps_bytes(), 0);
        s->tma = mlp_tma_prepare(hidden, members, s->wb.data(), s->maps.data());
    }
    if (!rc && s->tma && !std::getenv("MLSD_TRAIN_CUDA")) {
        // buffers of the tensor-core training step: transposed inputs, activations,
        // weights and gradients (rows of the transposes padded to a multiple of 8)
        SurTc &t = s->tc;
        t.max_rows = max_batch;
        t.ldT = (max_batch + 7) / 8 * 8;
        const size_t T = (size_t)t.ldT;
        void *p = nullptr;
        if (!rc) { rc = sur_alloc(s, &p, (size_t)MLSD_SUR_IN * T * 2); t.XT = (__nv_bfloat16 *)p; }
        for (int l = 0; l < 3 && !rc; ++l) { rc = sur_alloc(s, &p, H * T * 2); t.AT[l] = (__nv_bfloat16 *)p; }
        for (int l = 0; l < 2 && !rc; ++l) { rc = sur_alloc(s, &p, H * H * 2); t.WT[l] = (__nv_bfloat16 *)p; }
        for (int l = 0; l < 2 && !rc; ++l) { rc = sur_alloc(s, &p, M * H * 2); t.dZ[l] = (__nv_bfloat16 *)p; }
        for (int l = 0; l < 2 && !rc; ++l) { rc = sur_alloc(s, &p, H * T * 2); t.dZT[l] = (__nv_bfloat16 *)p; }
        s->train_tc = !rc;
    }
    if (rc) { mlsd_surrogate_free(s); return rc; }
    *out = s;
    return MLSD_OK;
}

int mlsd_surrogate_set_params(mlsd_surrogate *s, int member, const float *params_host)
{
    if (!s || member < 0 || member >= s->members || !params_host) return MLSD_EINVAL;
    const size_t np = (size_t)s->np;
    CK(cudaMemcpy(s->w[member], params_host, np * 4, cudaMemcpyHostToDevice));
    CK(cudaMemset(s->m[member], 0, np * 4));
    CK(cudaMemset(s->v[member], 0, np * 4));
    s->t[member] = 0;
    CK(sur_to_bf16(s->np, s->w[member], s->wb[member], nullptr));
    CK(cudaDeviceSynchronize());
    return MLSD_OK;
}

int mlsd_surrogate_get_params(mlsd_surrogate *s, int member, float *params_host)
{
    if (!s || member < 0 || member >= s->members || !params_host) return MLSD_EINVAL;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(params_host, s->w[member], (size_t)s->np * 4, cudaMemcpyDeviceToHost));
    return MLSD_OK;
}

int mlsd_surrogate_features(mlsd_levels *h, int level, const double *B_dev, void *X_dev,
                            float *F32_dev, void *cuda_stream)
{
    if (!h || level < 1 || level > h->L || !B_dev || !X_dev) return MLSD_EINVAL;
    DevLevel &d = h->lev[level - 1];
    if (d.cls.size() != 1 || !sur_size_ok(d.cls[0].n) || h->precision != MLSD_FP32)
        return MLSD_EUNSUPPORTED;
    const SizeClass &c = d.cls[0];
    CK(launch_features(static_cast<const float *>(c.band), c.Nl, c.tile, c.n, h->N, nullptr, h->P, B_dev,
                       h->kappa, X_dev, F32_dev, nullptr, static_cast<cudaStream_t>(cuda_stream)));
    return MLSD_OK;
}

int mlsd_surrogate_grad(mlsd_surrogate *s, int member, const void *X_dev, const float *Y_dev,
                        int M, float *grad_dev, double *loss_host, void *cuda_stream)
{
    if (!s || member < 0 || member >= s->members || !X_dev || !Y_dev || M < 1 || M > s->max_batch)
        return MLSD_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    CK(grad_of(s, member, M, X_dev, Y_dev,
                s->g[member], s->part, s->loss, s->ws, s->ws_n, st));
    if (grad_dev)
        CK(cudaMemcpyAsync(grad_dev, s->g[member], (size_t)s->np * 4, cudaMemcpyDeviceToDevice, st));
    if (loss_host) {
        CK(cudaMemcpyAsync(loss_host, s->loss, 8, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return MLSD_OK;
}

int mlsd_surrogate_train_step(mlsd_surrogate *s, int member, const void *X_dev,
                              const float *Y_dev, int M, float lr, double *loss_host,
                              void *cuda_stream)
{
    if (!s || member < 0 || member >= s->members || !X_dev || !Y_dev || M < 1 ||
        M > s->max_batch || !(lr > 0))
        return MLSD_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    CK(grad_of(s, member, M, X_dev, Y_dev,
                s->g[member], s->part, s->loss, s->ws, s->ws_n, st));
    s->t[member] += 1;
    CK(sur_adam(s->np, s->w[member], s->g[member], s->m[member], s->v[member], lr, s->t[member],
                s->wb[member], st));
    if (loss_host) {
        CK(cudaMemcpyAsync(loss_host, s->loss, 8, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return MLSD_OK;
}

int mlsd_surrogate_dataset(mlsd_levels *h, int level, const double *B_dev, void *X_dev, float *Y_dev,
                           void *cuda_stream)
{
    if (!h || level < 1 || level > h->L || !B_dev || !X_dev || !Y_dev) return MLSD_EINVAL;
    DevLevel &d = h->lev[level - 1];
    if (d.cls.size() != 1 || !sur_size_ok(d.cls[0].n) || h->precision != MLSD_FP32)
        return MLSD_EUNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const long long P = h->P;
    double *ws = nullptr;
    CK(cudaMallocAsync((void **)&ws, (size_t)P * 7 * 8, st));
    double *K = ws, *Q = ws + 3 * P;                 // Q: E and the series gap, [P][4]
    int rc = mlsd_solve_level(h, level, B_dev, K, nullptr, cuda_stream);
    cudaError_t e = cudaSuccess;
    const SizeClass &c = d.cls[0];
    if (!rc) e = launch_features(static_cast<const float *>(c.band), c.Nl, c.tile, c.n, h->N, nullptr, P, B_dev,
                                 h->kappa, X_dev, nullptr, Q, st);
    if (!rc && e == cudaSuccess) e = sur_targets(P, B_dev, K, Q, Y_dev, st);
    cudaFreeAsync(ws, st);
    if (rc) return rc;
    CK(e);
    return MLSD_OK;
}

namespace {
uint64_t splitmix64(uint64_t &x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
}  // namespace

int mlsd_surrogate_symmetry(const void *X_dev, const float *Y_dev, int64_t n_rows, int g,
                            void *X_out, float *Y_out, void *cuda_stream)
{
    if (n_rows < 0 || g < 0 || g > 7 || (!X_out && !Y_out) || (X_out && !X_dev) ||
        (Y_out && !Y_dev))
        return MLSD_EINVAL;
    CK(sur_symmetry(n_rows, g, X_dev, Y_dev, X_out, Y_out, static_cast<cudaStream_t>(cuda_stream)));
    return MLSD_OK;
}

int mlsd_surrogate_train(mlsd_surrogate *s, const void *X_dev, const float *Y_dev, int64_t n_rows,
                         int epochs, int batch, float lr, float lr_final, uint64_t seed,
                         int augment, double *losses_host, void *cuda_stream)
{
    const int64_t mult = augment ? 8 : 1;
    if (!s || !X_dev || !Y_dev || epochs < 1 || batch < 1 || batch > s->max_batch ||
        n_rows < 1 || n_rows * mult < batch || n_rows > (int64_t)0x7fffffff / mult ||
        !(lr > 0) || !(lr_final > 0))
        return MLSD_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int64_t rows = n_rows * mult;           // rows per epoch, images included
    const long long steps = rows / batch, total = steps * epochs;
    char *ws = nullptr;
    const size_t xb = (size_t)batch * MLSD_SUR_IN * 2, yb = (size_t)batch * 3 * 4, ib = (size_t)rows * 4;
    CK(cudaMallocAsync((void **)&ws, xb + yb + ib + 16, st));
    void *Xb = ws;
    float *Yb = reinterpret_cast<float *>(ws + xb);
    int *idx = reinterpret_cast<int *>(ws + xb + yb);
    double *acc = reinterpret_cast<double *>(ws + xb + yb + ((ib + 7) / 8) * 8);
    std::vector<int> perm((size_t)rows);
    cudaError_t e = cudaSuccess;
    for (int m = 0; m < s->members && e == cudaSuccess; ++m) {
        // each member its own shuffles: Fisher-Yates on a SplitMix64 stream
        uint64_t rs = seed * 0x9E3779B97F4A7C15ull + (uint64_t)m;
        long long t = 0;
        e = cudaMemsetAsync(acc, 0, 8, st);
        for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
            for (int64_t i = 0; i < rows; ++i) perm[(size_t)i] = (int)i;
            for (int64_t i = rows - 1; i > 0; --i) {
                const int64_t j = (int64_t)(splitmix64(rs) % (uint64_t)(i + 1));
                std::swap(perm[(size_t)i], perm[(size_t)j]);
            }
            e = cudaMemcpyAsync(idx, perm.data(), ib, cudaMemcpyHostToDevice, st);
            for (long long q = 0; q < steps && e == cudaSuccess; ++q, ++t) {
                const float r = lr * (float)std::pow((double)lr_final / lr, (double)t / (double)std::max(1LL, total - 1));
                e = sur_gather(batch, idx + q * batch, X_dev, Y_dev, Xb, Yb, augment ? 1 : 0, st);
                if (e == cudaSuccess)
                    e = grad_of(s, m, batch, Xb, Yb,
                                 s->g[m], s->part, s->loss, s->ws, s->ws_n, st);
                s->t[m] += 1;
                if (e == cudaSuccess)
                    e = sur_adam(s->np, s->w[m], s->g[m], s->m[m], s->v[m], r, s->t[m], s->wb[m], st);
                if (e == cudaSuccess && ep == epochs - 1) e = sur_add_loss(s->loss, acc, st);
            }
            // the host permutation buffer is refilled next epoch: the copy above must have
            // read it (pageable copies are staged before the call returns)
        }
        if (e == cudaSuccess && losses_host) {
            double a = 0.0;
            e = cudaMemcpyAsync(&a, acc, 8, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            losses_host[m] = a / (double)steps;
        }
    }
    cudaFreeAsync(ws, st);
    CK(e);
    return MLSD_OK;
}

int mlsd_surrogate_save(mlsd_surrogate *s, const char *path)
{
    if (!s || !path) return MLSD_EINVAL;
    std::vector<float> buf((size_t)s->np);
    FILE *f = std::fopen(path, "wb");
    if (!f) return MLSD_EINVAL;
    const char magic[8] = {'M', 'L', 'S', 'D', 'S', 'U', 'R', '1'};
    const int64_t hdr[3] = {s->members, s->h, s->np};
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, 8, 3, f) == 3;
    for (int m = 0; m < s->members && ok; ++m) {
        ok = mlsd_surrogate_get_params(s, m, buf.data()) == MLSD_OK &&
             std::fwrite(buf.data(), 4, buf.size(), f) == buf.size();
    }
    ok = (std::fclose(f) == 0) && ok;
    return ok ? MLSD_OK : MLSD_EINVAL;
}

int mlsd_surrogate_load(mlsd_surrogate *s, const char *path)
{
    if (!s || !path) return MLSD_EINVAL;
    FILE *f = std::fopen(path, "rb");
    if (!f) return MLSD_EINVAL;
    char magic[8];
    int64_t hdr[3];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "MLSDSUR1", 8) == 0 &&
              std::fread(hdr, 8, 3, f) == 3 && hdr[0] == s->members && hdr[1] == s->h && hdr[2] == s->np;
    std::vector<float> buf((size_t)s->np);
    for (int m = 0; m < s->members && ok; ++m)
        ok = std::fread(buf.data(), 4, buf.size(), f) == buf.size() &&
             mlsd_surrogate_set_params(s, m, buf.data()) == MLSD_OK;
    std::fclose(f);
    return ok ? MLSD_OK : MLSD_EINVAL;
}

int mlsd_surrogate_set_engine(mlsd_surrogate *s, int engine)
{
    if (!s || (engine != MLSD_SUR_CUDA && engine != MLSD_SUR_TENSOR)) return MLSD_EINVAL;
    if (engine == MLSD_SUR_TENSOR && !mlp_tc_supported(s->h)) return MLSD_EUNSUPPORTED;
    s->engine = engine;
    return MLSD_OK;
}

int mlsd_surrogate_status(mlsd_surrogate *s, void *cuda_stream)
{
    if (!s) return MLSD_EINVAL;
    CK(cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream)));
    int v = 0;
    CK(cudaMemcpy(&v, s->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (v) CK(cudaMemset(s->status, 0, sizeof(int)));
    return v;
}

int mlsd_surrogate_predict(mlsd_surrogate *s, const void *X_dev, int64_t M, float *out_dev,
                           void *cuda_stream)
{
    if (!s || !X_dev || !out_dev || M < 1) return MLSD_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (s->engine == MLSD_SUR_TENSOR) {
        if (s->tma && launch_mlp_tma(X_dev, M, s->h, s->members, s->maps.data(), s->wf_ptrs, out_dev,
                                     s->status, st) == cudaSuccess)
            return MLSD_OK;
        CK(launch_mlp_tc(X_dev, M, s->h, s->members, s->wb_ptrs, s->wf_ptrs, out_dev, s->status, st));
        return MLSD_OK;
    }
    const char *X = static_cast<const char *>(X_dev);
    for (int k = 0; k < s->members; ++k)
        for (int64_t r0 = 0; r0 < M; r0 += s->max_batch) {
            const int mb = (int)std::min<int64_t>(s->max_batch, M - r0);
            float *Z[4] = {s->Z[0], s->Z[1], s->Z[2], out_dev + ((size_t)k * M + r0) * 3};
            CK(sur_forward(s->h, mb, X + (size_t)r0 * MLSD_SUR_IN * 2, s->w[k], s->wb[k], Z, s->A,
                           s->ws, s->ws_n, st));
        }
    return MLSD_OK;
}

int mlsd_solve_level_surrogate(mlsd_levels *h, mlsd_surrogate *s, int level,
                               const double *K_base_dev, double *K_out_dev, double threshold,
                               int64_t *n_fallback_out, void *cuda_stream)
{
    if (!h || !s || level < 1 || level > h->L || !K_base_dev || !K_out_dev || !(threshold >= 0))
        return MLSD_EINVAL;
    DevLevel &d = h->lev[level - 1];
    if (d.cls.size() != 1 || !sur_size_ok(d.cls[0].n) || h->precision != MLSD_FP32)
        return MLSD_EUNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const long long P = h->P;
    char *ws = nullptr;
    const size_t xb = (size_t)P * MLSD_SUR_IN * 2, ob = (size_t)s->members * P * 3 * 4;
    const size_t fb = (size_t)P * 4, ib = (size_t)P * 4, qb = (size_t)P * 4 * 8;
    CK(cudaMallocAsync((void **)&ws, qb + xb + ob + fb + ib + 256, st));
    double *Q = reinterpret_cast<double *>(ws);
    void *X = ws + qb;
    float *out = reinterpret_cast<float *>(ws + qb + xb);
    int *flag = reinterpret_cast<int *>(ws + qb + xb + ob);
    int *idx = reinterpret_cast<int *>(ws + qb + xb + ob + fb);
    int *cnt = reinterpret_cast<int *>(ws + qb + xb + ob + fb + ib);
    int count = 0;
    const SizeClass &c0 = d.cls[0];
    int rc = MLSD_OK;
    cudaError_t e = launch_features(static_cast<const float *>(c0.band), c0.Nl, c0.tile, c0.n, h->N, nullptr,
                                    P, K_base_dev, h->kappa, X, nullptr, Q, st);
    if (e != cudaSuccess) rc = MLSD_ECUDA;
    if (!rc) rc = mlsd_surrogate_predict(s, X, P, out, cuda_stream);
    if (!rc) e = sur_disagree(P, s->members, out, K_base_dev, Q, threshold, K_out_dev, flag, idx, cnt, st);
    if (!rc && e == cudaSuccess) e = cudaMemcpyAsync(&count, cnt, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (!rc && e == cudaSuccess && count > 0) {
        // the plain patch solve on the flagged patches only; when they are too few to
        // fill the GPU their serial step latency decides, so take the tiling with the
        // most threads per patch field instead of the throughput-tuned one
        SizeClass fc = d.cls[0];
        fc.idx = idx;
        fc.count = count;
        int sms = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (count < sms) {
            std::vector<PatchVariant> vs;
            patch_variants(fc.n, h->precision, vs);
            for (auto &v : vs)
                if (!v.packed && !v.split && v.cluster == 1 && v.threads > fc.variant.threads) fc.variant = v;
        }
        PatchParams pp = patch_params(h, d, fc, K_base_dev, d.S, nullptr);
        e = launch_patch(fc.variant, pp, pp.items, st);
        if (e == cudaSuccess) e = sur_merge(count, idx, K_base_dev, d.S, K_out_dev, st);
    }
    cudaFreeAsync(ws, st);
    if (rc) return rc;
    CK(e);
    if (n_fallback_out) *n_fallback_out = count;
    return MLSD_OK;
}

}  // extern "C"

namespace {
// The surrogate's workspace for MLSD_SURROGATE chains, allocated with the handle
// (freed with it) when a surrogate is attached; reused on every chain.
int surrogate_workspace(mlsd_levels *h, DevLevel &d, mlsd_surrogate *sur)
{
    const long long P = h->P;
    int rc;
    if (!d.sur_E && (rc = dev_alloc(h, (void **)&d.sur_E, (size_t)P * 4 * 8))) return rc;
    if (!d.sur_X && (rc = dev_alloc(h, &d.sur_X, (size_t)P * MLSD_SUR_IN * 2))) return rc;
    if (!d.sur_flag && (rc = dev_alloc(h, (void **)&d.sur_flag, (size_t)P * 4))) return rc;
    if (!d.sur_idx && (rc = dev_alloc(h, (void **)&d.sur_idx, (size_t)P * 4))) return rc;
    if (!d.sur_cnt && (rc = dev_alloc(h, (void **)&d.sur_cnt, 16))) return rc;
    // the ensemble output grows with the member count of the attached surrogate
    static_assert(sizeof(float) == 4, "");
    const size_t ob = (size_t)sur->members * P * 3 * 4;
    if ((rc = dev_alloc(h, (void **)&d.sur_out, ob))) return rc;
    return MLSD_OK;
}

// One surrogate level on the stream with no host synchronisation: features and
// series estimates, the ensemble, the fallback rule with the compacted count
// left on the device, the plain patch solve of the flagged patches by a launch
// sized for every patch whose CTAs stride over the first 2 * count work items,
// and the merge of those solves into K*.
int surrogate_level_async(mlsd_levels *h, DevLevel &d, cudaStream_t st)
{
    mlsd_surrogate *sur = d.sur;
    const long long P = h->P;
    const SizeClass &c0 = d.cls[0];
    CK(launch_features(static_cast<const float *>(c0.band), c0.Nl, c0.tile, c0.n, h->N, nullptr, P,
                       d.base, h->kappa, d.sur_X, nullptr, d.sur_E, st));
    int rc = mlsd_surrogate_predict(sur, d.sur_X, P, d.sur_out, st);
    if (rc) return rc;
    CK(sur_disagree(P, sur->members, d.sur_out, d.base, d.sur_E, d.sur_thr, d.Kstar, d.sur_flag,
                    d.sur_idx, d.sur_cnt, st));
    PatchParams pp = patch_params(h, d, c0, d.base, d.S, nullptr);
    pp.pidx = d.sur_idx;
    pp.count_dev = d.sur_cnt;
    pp.item0 = 0;
    pp.items = 2 * P;
    int dev = 0, sms = 0, per_sm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c0.variant.fn, c0.variant.threads,
                                                     c0.variant.smem));
    // two waves of resident CTAs (in work items: packed kernels take two per CTA)
    const long long cap = 2LL * sms * std::max(per_sm, 1) * (c0.variant.packed ? 2 : 1);
    CK(launch_patch(c0.variant, pp, std::min<long long>(2 * P, cap), st));
    CK(sur_merge_dev(P, d.sur_cnt, d.sur_idx, d.base, d.S, d.Kstar, st));
    return MLSD_OK;
}
}  // namespace

extern "C" {

}  // extern "C"
