// Kernels of the batched patch solve (included by the translation units that
// instantiate them: patch_n32.cu, patch_n64.cu, patch_cluster.cu, and patch.cu
// for the shared device helpers).  Everything sits in an unnamed namespace:
// each unit compiles its own instantiations, which keeps the build parallel.
#pragma once
// Batched local patch solves: the numerical homogenization K[psi, B; Omega]
// of Sec. 2.2 (HMM steps 1-3) for every macro node of one level.
//
// One CTA advances one corrector field w_j of one patch (work item 2p + j - 1)
// for all its time steps with the whole field resident on chip:
//   * every thread owns a BX x BY block of cells and keeps w, the Heun stage
//     value and the two advection coefficients of its cells in registers;
//   * per RK stage the block edges go through shared memory (rows row-major,
//     columns in a transposed buffer, both 16-byte vectorised), one barrier
//     per stage (double-buffered exchange);
//   * the flux averages <v_i w_j> are summed in FP32 per thread over a window
//     of at most 32 steps and then added to FP64 accumulators; the CTA reduces
//     them in FP64 at the end.
// The stencil is the second-order central-difference operator
//   w_t = v1 (D0x w + d_j1) + v2 (D0y w + d_j2) + B11 Dxx w + 2 B12 Dxy w + B22 Dyy w
// with Dxy w = (D0x w(b+1) - D0x w(b-1)) / (2h), i.e. the E-W differences of
// the rows above and below, and Heun's RK2 w* = w + dt f(w),
// w <- (w + w* + dt f(w*)) / 2 with dt folded into the coefficients.
#include <cooperative_groups.h>
#include <cstdio>

#include "mlsd_internal.cuh"

namespace cg = cooperative_groups;

namespace mlsd {
namespace {

constexpr int kFlush = 32;   // FP32 flux partials are flushed to FP64 this often (steps)
constexpr long long kMaxSteps = 1ll << 30;   // larger step counts are rejected

template <typename T, int CNT>
__device__ __forceinline__ void st_vec(T *dst, const T (&src)[CNT])
{
    constexpr int bytes = CNT * (int)sizeof(T);
    if constexpr (bytes % 16 == 0) {
        constexpr int per = 16 / sizeof(T);
#pragma unroll
        for (int k = 0; k < CNT / per; ++k) {
            if constexpr (sizeof(T) == 4)
                reinterpret_cast<float4 *>(dst)[k] =
                    make_float4(src[4 * k], src[4 * k + 1], src[4 * k + 2], src[4 * k + 3]);
            else
                reinterpret_cast<double2 *>(dst)[k] = make_double2(src[2 * k], src[2 * k + 1]);
        }
    } else if constexpr (bytes % 8 == 0 && sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < CNT / 2; ++k)
            reinterpret_cast<float2 *>(dst)[k] = make_float2(src[2 * k], src[2 * k + 1]);
    } else {
#pragma unroll
        for (int k = 0; k < CNT; ++k) dst[k] = src[k];
    }
}

template <typename T, int CNT>
__device__ __forceinline__ void ld_vec(T (&dst)[CNT], const T *src, int off = 0)
{
    constexpr int bytes = CNT * (int)sizeof(T);
    if constexpr (bytes % 16 == 0) {
        constexpr int per = 16 / sizeof(T);
#pragma unroll
        for (int k = 0; k < CNT / per; ++k) {
            if constexpr (sizeof(T) == 4) {
                float4 v = reinterpret_cast<const float4 *>(src)[k];
                dst[off + 4 * k] = v.x; dst[off + 4 * k + 1] = v.y;
                dst[off + 4 * k + 2] = v.z; dst[off + 4 * k + 3] = v.w;
            } else {
                double2 v = reinterpret_cast<const double2 *>(src)[k];
                dst[off + 2 * k] = v.x; dst[off + 2 * k + 1] = v.y;
            }
        }
    } else if constexpr (bytes % 8 == 0 && sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < CNT / 2; ++k) {
            float2 v = reinterpret_cast<const float2 *>(src)[k];
            dst[off + 2 * k] = v.x; dst[off + 2 * k + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < CNT; ++k) dst[off + k] = src[k];
    }
}

// Shared-memory layout of one CTA.  A patch field of N x N cells is split over
// a cluster of C CTAs, each owning a slab of NS = N / C rows (C = 1: the whole
// field in one CTA).  Per RK stage every thread publishes the edges of its
// BX x BY block: top/bottom rows into row buffers (row-major), left/right
// columns into transposed column buffers whose stride is the slab height plus
// a 16-byte pad (conflict-free 128-bit transposed stores).  Double buffered.
template <int N, int C, int BX, int BY, typename real>
struct Smem {
    static constexpr int NS = N / C;
    static constexpr int NBX = N / BX, NBY = NS / BY;
    static constexpr int CS = NS + 16 / (int)sizeof(real);
    static constexpr int ROW = NBY * N;          // one row buffer (top or bottom edges)
    static constexpr int COL = NBX * CS;         // one column buffer (left or right edges)
    // C > 1: the neighbouring slabs' edge rows are pushed into HS (row below the
    // slab) and HN (row above) of this CTA before the stage barrier
    static constexpr int HALO = C > 1 ? 2 * N : 0;
    static constexpr int STAGE = 2 * ROW + 2 * COL + HALO;
    static constexpr int EXCH = 2 * STAGE;       // double buffered
    static constexpr int SETUP = N * (NS + 2);   // psi rows of the slab plus one halo row each side
    static constexpr int WORDS = (EXCH > SETUP ? EXCH : SETUP);
    static constexpr size_t BYTES = (size_t)WORDS * sizeof(real) + 64 * sizeof(double);
};

// Micro time step and window (same rules and operation order as the problem
// statement in mlsd.h): CFL on advection and diffusion, the RK2 stability cap,
// tau = L^2 / (4 pi^2 lambda_min).
__device__ void micro_schedule(double h, double L, double vmax, double B11, double B12,
                               double B22, double cfl, double t_burn, double t_avg,
                               long long nb_fixed, long long na_fixed, double &dt,
                               long long &nb, long long &na)
{
    double lmin = 0.5 * ((B11 + B22) - sqrt((B11 - B22) * (B11 - B22) + 4.0 * B12 * B12));
    double dd = h * h / (2.0 * (B11 + B22) + 4.0 * fabs(B12));
    dt = dd;
    if (vmax > 0.0) {
        double da = h / vmax;
        if (da < dt) dt = da;
    }
    dt *= cfl;
    if (vmax > 0.0) {
        double ds = cbrt(8.0 * lmin * h * h / (vmax * vmax * vmax * vmax));
        if (ds < dt) dt = ds;
    }
    double tau = L * L / (4.0 * kPi * kPi * lmin);
    const double fb = ceil(t_burn * tau / dt), fa = ceil(t_avg * tau / dt);
    // out-of-range counts (lmin <= 0, NaN) are mapped to -1 and rejected by the caller
    nb = (fb >= 0.0 && fb < 4.0e18) ? (long long)fb : -1;
    na = (fa >= 0.0 && fa < 4.0e18) ? (long long)fa : -1;
    if (na == 0) na = 1;
    if (!(lmin > 0.0)) { nb = -1; na = -1; }
    if (na_fixed > 0) { nb = nb_fixed; na = na_fixed; }
}

// CTA-level barrier, or cluster-wide (release/acquire) when the field is split
template <int C>
__device__ __forceinline__ void tile_sync()
{
    if constexpr (C == 1) __syncthreads();
    else cg::this_cluster().sync();
}

// shared memory of cluster rank r (the CTA's own when C == 1)
template <int C, typename T>
__device__ __forceinline__ T *rank_ptr(T *p, int r)
{
    if constexpr (C == 1) return p;
    else return cg::this_cluster().map_shared_rank(p, r);
}

// Uniform coefficients of one stage, from dt, h and the base tensor B:
// b_ii = dt B_ii / h^2, bx = dt B12 / (2 h^2), bc = 1 - 2 (b11 + b22), and the
// constant part K = -2h b_JJ of the source term of field J.
template <typename real>
struct Coef {
    real b11x2, b22x2, bx, bc, twoh, K, halfK;
};

// Neighbour signalling for cluster-split fields (SYNC = 2).  A thread that
// pushed a slab edge row into a neighbour's halo slot arrives on that
// neighbour's mbarrier for the stage buffer (release at cluster scope); the
// threads that read the halo slots wait on their own CTA's mbarrier (acquire).
__device__ __forceinline__ void nbr_arrive(uint32_t mbar_local, int rank)
{
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(mbar_local), "r"(rank));
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" :: "r"(remote)
                 : "memory");
}

// Bounded wait for the phase of the given parity: false after about a second
// (2^31 SM clocks), or after about half a millisecond (2^20 clocks) when another
// wait of the launch has already timed out (status holds MLSD_ETIMEOUT), so that
// a failed exchange ends the launch quickly instead of costing every remaining
// CTA a full second.  The status word (global memory) is not read in the first
// 2^20 clocks: an ordinary wait for a neighbour's rows lasts a few microseconds,
// and a global load per retry would delay the retry that sees the phase complete.
__device__ __forceinline__ bool nbr_wait(uint32_t mbar_local, uint32_t parity, const int *status)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok) : "r"(mbar_local), "r"(parity) : "memory");
        if (ok) return true;
        const long long dt = clock64() - t0;
        if (dt > (1ll << 31)) return false;
        if (dt > (1ll << 20) && *(volatile const int *)status == MLSD_ETIMEOUT) return false;
    }
}

// Bulk copy (async proxy) of `bytes` from this CTA's shared memory to the
// shared memory of cluster rank `rank`, completing on that rank's mbarrier at
// the same offset as `mbar_local` (SYNC = 3).
__device__ __forceinline__ void bulk_to_rank(uint32_t dst_local, uint32_t src_local, uint32_t bytes,
                                             uint32_t mbar_local, int rank)
{
    uint32_t dst, mbar;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(dst) : "r"(dst_local), "r"(rank));
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(mbar) : "r"(mbar_local), "r"(rank));
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "r"(src_local), "r"(bytes), "r"(mbar) : "memory");
}

// arm the next phase of a local mbarrier: one arrival plus `bytes` expected
__device__ __forceinline__ void arm_tx(uint32_t mbar_local, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar_local), "r"(bytes)
                 : "memory");
}

// Coef as f32x2 pairs (both lanes equal) for the row-paired kernel (SYNC = 4)
struct CoefP {
    float2 b11x2, b22x2, bx, bc, T, K, halfK;
};

// ---------------------------------------------------------------------------
// Stencil coefficients in tensor memory (the "t" tilings: FP32, 4 x 8 cells per
// thread).  The two per-cell coefficients aE, aN of a thread's block (64 words)
// live in the SM's tensor memory instead of its registers, so that a cell needs
// only two registers (w and the stage value): a field then takes half the
// register file it takes otherwise, and a 128^2 field fits one CTA of 512
// threads, a 256^2 field a cluster of 4.  Warp w may address only the TMEM
// lanes 32 (w % 4) .. +31; its threads own those lanes (one each) and the
// columns 64 (w / 4) .. +63, block row r at columns 8 r .. 8 r + 7 as
// (aE[0..3], aN[0..3]).  A CTA of NT threads allocates NT / 2 columns.  Every
// such kernel holds at least 64 registers per thread (w and the stage value of
// 32 cells), so the CTAs that fit an SM's register file (65536 registers) ask
// for at most 65536 / 128 = 512 columns, the SM's whole tensor memory: an
// allocation never waits on another CTA of these kernels.
__device__ __forceinline__ void tm_st8(uint32_t taddr, const float (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :: "r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])),
                    "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
                    "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                    "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}

__device__ __forceinline__ void tm_wait_st()
{
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// start loading 8 columns of this thread's lane; the values are valid after tm_wait_ld
__device__ __forceinline__ void tm_ld8(uint32_t taddr, uint32_t (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
}

// wait for this thread's outstanding tensor-memory loads; the registers of the
// last load pass through the statement, so no use of them is placed before it
__device__ __forceinline__ void tm_wait_ld(uint32_t (&v)[8])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]),
                   "+r"(v[6]), "+r"(v[7]));
}

template <int N, int C, int BX, int BY, typename real>
struct Tile {
    using S = Smem<N, C, BX, BY, real>;
    static constexpr int NS = S::NS, NBX = S::NBX, NBY = S::NBY, NT = NBX * NBY;

    // Barrier over the threads that share this field.  GR = false: the CTA.
    // GR = true (one field per group of NT threads of a larger CTA, C = 1): the
    // group, by a named barrier (ids 1.., one per group of NT >= 64 threads) or,
    // for one-warp groups, __syncwarp.
    template <bool GR>
    __device__ __forceinline__ static void csync()
    {
        if constexpr (!GR) {
            __syncthreads();
        } else if constexpr (NT == 32) {
            __syncwarp();
        } else {
            static_assert(NT % 32 == 0 && C == 1, "groups of whole warps, one CTA per field");
            asm volatile("bar.sync %0, %1;" :: "r"(1 + (int)(threadIdx.x / NT)), "r"(NT) : "memory");
        }
    }

    // Publish the edges of x into buffer `buf`; with a cluster, also push the
    // slab's first row into the HN slot of the rank below (its row above) and the
    // slab's last row into the HS slot of the rank above (its row below).
    // PUSH = false: local buffers only (the slab's first and last rows are then
    // moved by bulk copies, see stage()).
    template <bool PUSH = true>
    __device__ __forceinline__ static void publish_edges(real *sm, int buf, int rank, int tx, int ty,
                                                         const real (&x)[BY][BX])
    {
        const int a0 = tx * BX, b0 = ty * BY;
        real *rowT = sm + buf * S::STAGE;
        real *rowB = rowT + S::ROW;
        real *colL = rowB + S::ROW;
        real *colR = colL + S::COL;
        real t[BX], bt[BX];
#pragma unroll
        for (int c = 0; c < BX; ++c) { t[c] = x[0][c]; bt[c] = x[BY - 1][c]; }
        st_vec<real, BX>(rowT + ty * N + a0, t);
        st_vec<real, BX>(rowB + ty * N + a0, bt);
        real l[BY], r[BY];
#pragma unroll
        for (int k = 0; k < BY; ++k) { l[k] = x[k][0]; r[k] = x[k][BX - 1]; }
        st_vec<real, BY>(colL + tx * S::CS + b0, l);
        st_vec<real, BY>(colR + tx * S::CS + b0, r);
        if constexpr (C > 1 && PUSH) {
            real *HS = colR + S::COL, *HN = HS + N;
            if (ty == NBY - 1) st_vec<real, BX>(rank_ptr<C>(HS + a0, (rank + 1) % C), bt);
            if (ty == 0) st_vec<real, BX>(rank_ptr<C>(HN + a0, (rank + C - 1) % C), t);
        }
    }

    // halos of block (tx, ty) from buffer `buf`, all local after the barrier
    __device__ __forceinline__ static void load_halos(real *sm, int buf, int tx, int ty,
                                                      real (&hS)[BX], real (&hN)[BX],
                                                      real (&hW)[BY + 2], real (&hE)[BY + 2])
    {
        const int a0 = tx * BX, b0 = ty * BY;
        real *rowT = sm + buf * S::STAGE;
        real *rowB = rowT + S::ROW;
        real *colL = rowB + S::ROW;
        real *colR = colL + S::COL;
        const int tyS = (ty + NBY - 1) % NBY, tyN = (ty + 1) % NBY;
        const int txW = (tx + NBX - 1) % NBX, txE = (tx + 1) % NBX;
        const real *cw = colR + txW * S::CS;
        const real *ce = colL + txE * S::CS;
        real tmpw[BY], tmpe[BY];
        ld_vec<real, BY>(tmpw, cw + b0);
        ld_vec<real, BY>(tmpe, ce + b0);
#pragma unroll
        for (int k = 0; k < BY; ++k) { hW[k + 1] = tmpw[k]; hE[k + 1] = tmpe[k]; }
        const int aw = (a0 + N - 1) % N, ae = (a0 + BX) % N;
        if (C > 1 && ty == 0) {
            const real *HS = colR + S::COL;
            ld_vec<real, BX>(hS, HS + a0);
            hW[0] = HS[aw]; hE[0] = HS[ae];
        } else {
            ld_vec<real, BX>(hS, rowB + tyS * N + a0);
            const int bs = (b0 + NS - 1) % NS;
            hW[0] = cw[bs]; hE[0] = ce[bs];
        }
        if (C > 1 && ty == NBY - 1) {
            const real *HN = colR + S::COL + N;
            ld_vec<real, BX>(hN, HN + a0);
            hW[BY + 1] = HN[aw]; hE[BY + 1] = HN[ae];
        } else {
            ld_vec<real, BX>(hN, rowT + tyN * N + a0);
            const int bn = (b0 + BY) % NS;
            hW[BY + 1] = cw[bn]; hE[BY + 1] = ce[bn];
        }
    }

    // SYNC = 3 (clusters): after the block edges of buffer `buf` are in shared
    // memory, the slab's last row goes to rank + 1's HS slot and its first row to
    // rank - 1's HN slot by two bulk copies issued by thread 0, each completing on
    // the receiver's mbarrier of this buffer; the rows written by the threads must
    // reach the async proxy first.  The source rows are not rewritten before both
    // copies have landed: the receivers wait for them before they send the next
    // stage's rows.  Only the threads on the slab's first and last block rows wait
    // for the incoming rows.
    __device__ __forceinline__ static void bulk_rows(real *sm, int buf, int rank, int tx, int ty,
                                                     uint32_t mbar, uint32_t parity, int *status,
                                                     bool *live)
    {
        if (ty == 0 || ty == NBY - 1) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tx == 0 && ty == 0 && *live) {
            real *rowT = sm + buf * S::STAGE, *rowB = rowT + S::ROW;
            real *HS = rowB + S::ROW + 2 * S::COL, *HN = HS + N;
            const uint32_t bytes = (uint32_t)(N * sizeof(real));
            bulk_to_rank((uint32_t)__cvta_generic_to_shared(HS),
                         (uint32_t)__cvta_generic_to_shared(rowB + (NBY - 1) * N), bytes, mbar,
                         (rank + 1) % C);
            bulk_to_rank((uint32_t)__cvta_generic_to_shared(HN),
                         (uint32_t)__cvta_generic_to_shared(rowT), bytes, mbar, (rank + C - 1) % C);
        }
        if ((ty == 0 || ty == NBY - 1) && *live) {
            if (!nbr_wait(mbar, parity, status)) {
                *live = false;
                atomicCAS(status, 0, MLSD_ETIMEOUT);
            } else if (tx == 0 && ty == 0) {
                // the phase completed: thread 0 re-arms this buffer's barrier
                arm_tx(mbar, (uint32_t)(2 * N * sizeof(real)));
            }
        }
    }

    // Exchange the edges of x through buffer `buf`, then form x + dt f(x),
    //   bc x + b11 (xE + xW) + b22 (xN + xS) + A1 (xE - xW) + A2 (xN - xS)
    //      + 2h A_J + bx (dEW(b+1) - dEW(b-1)),
    // with the per-cell coefficients aE = A1 + b11, aN = A2 + b22 (Coef):
    //   aE (xE - xW) + 2 b11 xW = A1 (xE - xW) + b11 (xE + xW), likewise in x2, and
    //   the source 2h A_J = 2h a_J - 2h b_JJ, whose constant part is Coef::K.
    // Ten FP32 instructions per cell.  SECOND: out = (w + g) / 2, with w (held in
    // out) seeding the FMA chain and K / 2 added by the final FMA.
    //
    // SYNC = 0: one cluster-wide (C = 1: CTA) barrier after the edges are out.
    // SYNC = 2: a CTA barrier for the in-slab halos, and neighbour signalling
    // (mbarrier `mbar` of this buffer, phase `parity`) for the two halo rows
    // that come from the neighbouring slabs; only the threads on the slab's
    // first and last block rows wait for those.
    //
    // SYNC = 2, 3 after a timeout: `live` (per thread) turns false when this
    // thread's wait runs out; the thread then waits no more, and thread 0 stops
    // re-arming the barriers and issuing bulk copies.  The neighbours' waits run
    // out in turn (within half a millisecond once the status word holds
    // MLSD_ETIMEOUT), so every rank finishes its remaining steps without waiting
    // and the ranks meet at the cluster barriers after the loop.
    template <int J, bool SECOND, int SYNC = 0>
    __device__ __forceinline__ static void stage(real *sm, int buf, int rank, int tx, int ty,
                                                 const real (&x)[BY][BX], real (&out)[BY][BX],
                                                 const real (&aE)[BY][BX], const real (&aN)[BY][BX],
                                                 const Coef<real> &k, uint32_t mbar = 0,
                                                 uint32_t parity = 0, int *status = nullptr,
                                                 bool *live = nullptr)
    {
        if constexpr (SYNC == 5 && C > 1) {
            stage_defer<J, SECOND>(sm, buf, rank, tx, ty, x, out, aE, aN, k, mbar, parity, status,
                                   live);
            return;
        }
        publish_edges<SYNC != 3>(sm, buf, rank, tx, ty, x);
        if constexpr (SYNC == 3 && C > 1) {
            bulk_rows(sm, buf, rank, tx, ty, mbar, parity, status, live);
        } else if constexpr (SYNC == 2 && C > 1) {
            if (ty == NBY - 1) nbr_arrive(mbar, (rank + 1) % C);       // its HS slot
            if (ty == 0) nbr_arrive(mbar, (rank + C - 1) % C);         // its HN slot
            __syncthreads();
            if ((ty == 0 || ty == NBY - 1) && *live)
                if (!nbr_wait(mbar, parity, status)) {
                    *live = false;
                    atomicCAS(status, 0, MLSD_ETIMEOUT);
                }
        } else {
            tile_sync<C>();
        }
        // halos: south row b0-1, north row b0+BY, west column a0-1, east column a0+BX
        real hS[BX], hN[BX], hW[BY + 2], hE[BY + 2];
        load_halos(sm, buf, tx, ty, hS, hN, hW, hE);
        // rolling E-W differences of rows r-1, r, r+1
        real dm[BX], d0[BX], dp[BX];
#pragma unroll
        for (int c = 0; c < BX; ++c) {
            real e = (c + 1 < BX) ? hS[c + 1] : hE[0];
            real w = (c > 0) ? hS[c - 1] : hW[0];
            dm[c] = e - w;
            real e0 = (c + 1 < BX) ? x[0][c + 1] : hE[1];
            real w0 = (c > 0) ? x[0][c - 1] : hW[1];
            d0[c] = e0 - w0;
        }
#pragma unroll
        for (int r = 0; r < BY; ++r) {
#pragma unroll
            for (int c = 0; c < BX; ++c) {
                real e, w;
                if (r + 1 < BY) {
                    e = (c + 1 < BX) ? x[r + 1][c + 1] : hE[r + 2];
                    w = (c > 0) ? x[r + 1][c - 1] : hW[r + 2];
                } else {
                    e = (c + 1 < BX) ? hN[c + 1] : hE[BY + 1];
                    w = (c > 0) ? hN[c - 1] : hW[BY + 1];
                }
                dp[c] = e - w;
            }
#pragma unroll
            for (int c = 0; c < BX; ++c) {
                const real xc = x[r][c];
                const real xE = (c + 1 < BX) ? x[r][c + 1] : hE[r + 1];
                const real xW = (c > 0) ? x[r][c - 1] : hW[r + 1];
                const real xN = (r + 1 < BY) ? x[r + 1][c] : hN[c];
                const real xS = (r > 0) ? x[r - 1][c] : hS[c];
                (void)xE;
                cell<J, SECOND>(out[r][c], xc, xW, xN, xS, d0[c], dm[c], dp[c], aE[r][c],
                                aN[r][c], k);
            }
#pragma unroll
            for (int c = 0; c < BX; ++c) { dm[c] = d0[c]; d0[c] = dp[c]; }
        }
    }

    // stage() with the per-cell coefficients in tensor memory (the "t" tilings):
    // `tcol` addresses this thread's first column.  Each row's coefficients are
    // loaded just before the row (loading them one row ahead measured no
    // faster); the arithmetic and its order are those of stage(), so both give
    // the same bits for the same block shape.  SYNC = 0 (one barrier per stage)
    // or 3 (bulk row copies between the slabs of a cluster).  FLUX (second stage
    // of a step inside the averaging window): the flux sums q1 += aE w,
    // q2 += aN w, qw += w of the new values are formed here, in stage()'s cell
    // order, from the coefficients already loaded.  LZ: the west and east halo
    // columns are read in pairs of rows as the row loop reaches them instead of
    // all at once, so that fewer of them are live (the values are
    // load_halos()').  GR: the field is one of a CTA's groups (see run()).
    template <int J, bool SECOND, int SYNC, bool FLUX = false, bool LZ = false, bool GR = false>
    __device__ __forceinline__ static void stage_tm(real *sm, int buf, int rank, int tx, int ty,
                                                    const real (&x)[BY][BX], real (&out)[BY][BX],
                                                    uint32_t tcol, const Coef<real> &k, uint32_t mbar,
                                                    uint32_t parity, int *status, bool *live,
                                                    real &q1, real &q2, real &qw)
    {
        static_assert(BX == 4 && BY == 8 && sizeof(real) == 4, "coefficient rows of 8 words");
        static_assert(SYNC == 0 || (SYNC == 3 && C > 1), "barrier per stage or bulk row copies");
        publish_edges<SYNC != 3>(sm, buf, rank, tx, ty, x);
        if constexpr (SYNC == 3) bulk_rows(sm, buf, rank, tx, ty, mbar, parity, status, live);
        else if constexpr (C > 1) tile_sync<C>();
        else csync<GR>();
        real hS[BX], hN[BX], hW[BY + 2], hE[BY + 2];
        const real *cw = nullptr, *ce = nullptr;      // LZ: this block's rows of the column halos
        if constexpr (LZ) {
            const int a0 = tx * BX, b0 = ty * BY;
            real *rowT = sm + buf * S::STAGE;
            real *rowB = rowT + S::ROW;
            real *colL = rowB + S::ROW;
            real *colR = colL + S::COL;
            const int tyS = (ty + NBY - 1) % NBY, tyN = (ty + 1) % NBY;
            const int txW = (tx + NBX - 1) % NBX, txE = (tx + 1) % NBX;
            const real *cwc = colR + txW * S::CS, *cec = colL + txE * S::CS;
            cw = cwc + b0;
            ce = cec + b0;
            const int aw = (a0 + N - 1) % N, ae = (a0 + BX) % N;
            if (C > 1 && ty == 0) {
                const real *HS = colR + S::COL;
                ld_vec<real, BX>(hS, HS + a0);
                hW[0] = HS[aw]; hE[0] = HS[ae];
            } else {
                ld_vec<real, BX>(hS, rowB + tyS * N + a0);
                const int bs = (b0 + NS - 1) % NS;
                hW[0] = cwc[bs]; hE[0] = cec[bs];
            }
            if (C > 1 && ty == NBY - 1) {
                const real *HN = colR + S::COL + N;
                ld_vec<real, BX>(hN, HN + a0);
                hW[BY + 1] = HN[aw]; hE[BY + 1] = HN[ae];
            } else {
                ld_vec<real, BX>(hN, rowT + tyN * N + a0);
                const int bn = (b0 + BY) % NS;
                hW[BY + 1] = cwc[bn]; hE[BY + 1] = cec[bn];
            }
            // rows b0, b0 + 1 (16-byte aligned column buffers: cw + 2i is 8-byte aligned)
            const float2 w2 = *reinterpret_cast<const float2 *>(cw);
            const float2 e2 = *reinterpret_cast<const float2 *>(ce);
            hW[1] = w2.x; hW[2] = w2.y; hE[1] = e2.x; hE[2] = e2.y;
        } else {
            load_halos(sm, buf, tx, ty, hS, hN, hW, hE);
        }
        uint32_t cv[8];
        __syncwarp();
        real dm[BX], d0[BX], dp[BX];
#pragma unroll
        for (int c = 0; c < BX; ++c) {
            real e = (c + 1 < BX) ? hS[c + 1] : hE[0];
            real w = (c > 0) ? hS[c - 1] : hW[0];
            dm[c] = e - w;
            real e0 = (c + 1 < BX) ? x[0][c + 1] : hE[1];
            real w0 = (c > 0) ? x[0][c - 1] : hW[1];
            d0[c] = e0 - w0;
        }
#pragma unroll
        for (int r = 0; r < BY; ++r) {
            if constexpr (LZ) {
                if ((r & 1) && r + 2 <= BY) {               // rows b0 + r + 1, b0 + r + 2
                    const float2 w2 = *reinterpret_cast<const float2 *>(cw + r + 1);
                    const float2 e2 = *reinterpret_cast<const float2 *>(ce + r + 1);
                    hW[r + 2] = w2.x; hW[r + 3] = w2.y; hE[r + 2] = e2.x; hE[r + 3] = e2.y;
                }
            }
            tm_ld8(tcol + 8 * r, cv);
            tm_wait_ld(cv);
#pragma unroll
            for (int c = 0; c < BX; ++c) {
                real e, w;
                if (r + 1 < BY) {
                    e = (c + 1 < BX) ? x[r + 1][c + 1] : hE[r + 2];
                    w = (c > 0) ? x[r + 1][c - 1] : hW[r + 2];
                } else {
                    e = (c + 1 < BX) ? hN[c + 1] : hE[BY + 1];
                    w = (c > 0) ? hN[c - 1] : hW[BY + 1];
                }
                dp[c] = e - w;
            }
#pragma unroll
            for (int c = 0; c < BX; ++c) {
                const real xc = x[r][c];
                const real xW = (c > 0) ? x[r][c - 1] : hW[r + 1];
                const real xN = (r + 1 < BY) ? x[r + 1][c] : hN[c];
                const real xS = (r > 0) ? x[r - 1][c] : hS[c];
                const real aE = __uint_as_float(cv[c]), aN = __uint_as_float(cv[4 + c]);
                cell<J, SECOND>(out[r][c], xc, xW, xN, xS, d0[c], dm[c], dp[c], aE, aN, k);
            }
            if constexpr (FLUX) {
#pragma unroll
                for (int c = 0; c < BX; ++c) {
                    q1 = fma(__uint_as_float(cv[c]), out[r][c], q1);
                    q2 = fma(__uint_as_float(cv[4 + c]), out[r][c], q2);
                    qw += out[r][c];
                }
            }
#pragma unroll
            for (int c = 0; c < BX; ++c) { dm[c] = d0[c]; d0[c] = dp[c]; }
        }
    }

    // E-W difference of row r of x (r = 0 .. BY-1) with the block's column halos
    __device__ __forceinline__ static void row_diff(real (&d)[BX], const real (&x)[BY][BX], int r,
                                                    const real (&hW)[BY + 2], const real (&hE)[BY + 2])
    {
#pragma unroll
        for (int c = 0; c < BX; ++c) {
            const real e = (c + 1 < BX) ? x[r][c + 1] : hE[r + 1];
            const real w = (c > 0) ? x[r][c - 1] : hW[r + 1];
            d[c] = e - w;
        }
    }

    // E-W difference of a halo row h (the row below, corner = 0, or above, corner = BY + 1)
    __device__ __forceinline__ static void halo_diff(real (&d)[BX], const real (&h)[BX], int corner,
                                                     const real (&hW)[BY + 2], const real (&hE)[BY + 2])
    {
#pragma unroll
        for (int c = 0; c < BX; ++c) {
            const real e = (c + 1 < BX) ? h[c + 1] : hE[corner];
            const real w = (c > 0) ? h[c - 1] : hW[corner];
            d[c] = e - w;
        }
    }

    // Stage with bulk row copies and the cross-slab rows deferred (SYNC = 5).  As
    // SYNC = 3, thread 0 sends the slab's first and last rows to the neighbouring
    // ranks by bulk copies right after the CTA barrier; but every thread first
    // computes the rows of its block that need no row halo (rows 1 .. BY-2: the
    // column halos come from this CTA), and only then do the slab-edge threads
    // wait for the incoming rows.  The copies' latency is spent on (BY-2)/BY of
    // the stage's arithmetic.  Rows BY-1 and 0 follow, the latter with its E-W
    // differences of rows 0 and 1 formed again (BX subtractions each).  The
    // arithmetic per cell is that of stage().
    template <int J, bool SECOND>
    __device__ __forceinline__ static void stage_defer(real *sm, int buf, int rank, int tx, int ty,
                                                       const real (&x)[BY][BX], real (&out)[BY][BX],
                                                       const real (&aE)[BY][BX], const real (&aN)[BY][BX],
                                                       const Coef<real> &k, uint32_t mbar, uint32_t parity,
                                                       int *status, bool *live)
    {
        static_assert(BY >= 2, "deferred rows need two rows per block");
        publish_edges<false>(sm, buf, rank, tx, ty, x);
        const bool edge = ty == 0 || ty == NBY - 1;
        if (edge) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        real *rowT = sm + buf * S::STAGE, *rowB = rowT + S::ROW;
        real *colL = rowB + S::ROW, *colR = colL + S::COL;
        real *HS = colR + S::COL, *HN = HS + N;
        if (tx == 0 && ty == 0 && *live) {
            const uint32_t bytes = (uint32_t)(N * sizeof(real));
            bulk_to_rank((uint32_t)__cvta_generic_to_shared(HS),
                         (uint32_t)__cvta_generic_to_shared(rowB + (NBY - 1) * N), bytes, mbar,
                         (rank + 1) % C);
            bulk_to_rank((uint32_t)__cvta_generic_to_shared(HN),
                         (uint32_t)__cvta_generic_to_shared(rowT), bytes, mbar, (rank + C - 1) % C);
        }
        const int a0 = tx * BX, b0 = ty * BY;
        const int txW = (tx + NBX - 1) % NBX, txE = (tx + 1) % NBX;
        const real *cw = colR + txW * S::CS, *ce = colL + txE * S::CS;
        // column halos of rows 0 .. BY-1 (this CTA's buffers)
        real hW[BY + 2], hE[BY + 2];
        {
            real tmpw[BY], tmpe[BY];
            ld_vec<real, BY>(tmpw, cw + b0);
            ld_vec<real, BY>(tmpe, ce + b0);
#pragma unroll
            for (int r = 0; r < BY; ++r) { hW[r + 1] = tmpw[r]; hE[r + 1] = tmpe[r]; }
        }
        // rows 1 .. BY-2
        real dm[BX], d0[BX], dp[BX];
        row_diff(dm, x, 0, hW, hE);
        row_diff(d0, x, 1, hW, hE);
#pragma unroll
        for (int r = 1; r < BY - 1; ++r) {
            row_diff(dp, x, r + 1, hW, hE);
#pragma unroll
            for (int c = 0; c < BX; ++c) {
                const real xW = (c > 0) ? x[r][c - 1] : hW[r + 1];
                cell<J, SECOND>(out[r][c], x[r][c], xW, x[r + 1][c], x[r - 1][c], d0[c], dm[c], dp[c],
                                aE[r][c], aN[r][c], k);
            }
#pragma unroll
            for (int c = 0; c < BX; ++c) { dm[c] = d0[c]; d0[c] = dp[c]; }
        }
        // now dm, d0 hold the differences of rows BY-2, BY-1; the row halos
        if (edge && *live) {
            if (!nbr_wait(mbar, parity, status)) {
                *live = false;
                atomicCAS(status, 0, MLSD_ETIMEOUT);
            } else if (tx == 0 && ty == 0) {
                arm_tx(mbar, (uint32_t)(2 * N * sizeof(real)));
            }
        }
        const int aw = (a0 + N - 1) % N, ae = (a0 + BX) % N;
        real hN[BX];
        if (ty == NBY - 1) {
            ld_vec<real, BX>(hN, HN + a0);
            hW[BY + 1] = HN[aw]; hE[BY + 1] = HN[ae];
        } else {
            ld_vec<real, BX>(hN, rowT + (ty + 1) * N + a0);
            const int bn = b0 + BY;
            hW[BY + 1] = cw[bn]; hE[BY + 1] = ce[bn];
        }
        // row BY-1
        halo_diff(dp, hN, BY + 1, hW, hE);
#pragma unroll
        for (int c = 0; c < BX; ++c) {
            const real xW = (c > 0) ? x[BY - 1][c - 1] : hW[BY];
            cell<J, SECOND>(out[BY - 1][c], x[BY - 1][c], xW, hN[c], x[BY - 2][c], d0[c], dm[c],
                            dp[c], aE[BY - 1][c], aN[BY - 1][c], k);
        }
        real hS[BX];
        if (ty == 0) {
            ld_vec<real, BX>(hS, HS + a0);
            hW[0] = HS[aw]; hE[0] = HS[ae];
        } else {
            ld_vec<real, BX>(hS, rowB + (ty - 1) * N + a0);
            const int bs = b0 - 1;
            hW[0] = cw[bs]; hE[0] = ce[bs];
        }
        // row 0
        halo_diff(dm, hS, 0, hW, hE);
        row_diff(d0, x, 0, hW, hE);
        row_diff(dp, x, 1, hW, hE);
#pragma unroll
        for (int c = 0; c < BX; ++c) {
            const real xW = (c > 0) ? x[0][c - 1] : hW[1];
            cell<J, SECOND>(out[0][c], x[0][c], xW, x[1][c], hS[c], d0[c], dm[c], dp[c], aE[0][c],
                            aN[0][c], k);
        }
    }

    // One cell of a stage (see stage()): dEW = xE - xW of this row, dm / dp those
    // of the rows below / above; o holds w on entry when SECOND.
    template <int J, bool SECOND>
    __device__ __forceinline__ static void cell(real &o, real xc, real xW, real xN, real xS,
                                                real dEW, real dm, real dp, real aE, real aN,
                                                const Coef<real> &k)
    {
        real d1 = dEW, d2 = xN - xS;
        if constexpr (J == 1) d1 = d1 + k.twoh; else d2 = d2 + k.twoh;
        const real cr = dp - dm;
        real g = fma(aE, d1, SECOND ? o : k.K);
        g = fma(k.b11x2, xW, g);
        g = fma(aN, d2, g);
        g = fma(k.b22x2, xS, g);
        g = fma(k.bx, cr, g);
        g = fma(k.bc, xc, g);
        o = SECOND ? fma(g, (real)0.5, k.halfK) : g;
    }

    // Split-phase stage.  On entry x's edges are in buffer `buf` and this thread
    // has arrived at the stage barrier.  Interior cells (no halo needed) are
    // computed while the barrier completes; then the halos are read and the
    // boundary ring is computed; finally out's edges go to buffer buf ^ 1 and
    // the thread arrives for the next stage.

    template <int J, bool SECOND>
    __device__ __forceinline__ static void stage_split(real *sm, int buf, int rank, int tx, int ty,
                                                       const real (&x)[BY][BX], real (&out)[BY][BX],
                                                       const real (&aE)[BY][BX], const real (&aN)[BY][BX],
                                                       const Coef<real> &k)
    {
        // ---- interior: rows 1..BY-2, columns 1..BX-2 (rolling E-W differences) ----
        {
            real dm[BX], d0[BX], dp[BX];
#pragma unroll
            for (int c = 1; c < BX - 1; ++c) { dm[c] = x[0][c + 1] - x[0][c - 1]; d0[c] = x[1][c + 1] - x[1][c - 1]; }
#pragma unroll
            for (int r = 1; r < BY - 1; ++r) {
#pragma unroll
                for (int c = 1; c < BX - 1; ++c) dp[c] = x[r + 1][c + 1] - x[r + 1][c - 1];
#pragma unroll
                for (int c = 1; c < BX - 1; ++c)
                    cell<J, SECOND>(out[r][c], x[r][c], x[r][c - 1], x[r + 1][c], x[r - 1][c],
                                    d0[c], dm[c], dp[c], aE[r][c], aN[r][c], k);
#pragma unroll
                for (int c = 1; c < BX - 1; ++c) { dm[c] = d0[c]; d0[c] = dp[c]; }
            }
        }
        asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
        real hS[BX], hN[BX], hW[BY + 2], hE[BY + 2];
        load_halos(sm, buf, tx, ty, hS, hN, hW, hE);
        // x with halos: X(r, c) for r = -1..BY, c = -1..BX
        auto X = [&](int r, int c) -> real {
            if (r < 0) return c < 0 ? hW[0] : (c >= BX ? hE[0] : hS[c]);
            if (r >= BY) return c < 0 ? hW[BY + 1] : (c >= BX ? hE[BY + 1] : hN[c]);
            return c < 0 ? hW[r + 1] : (c >= BX ? hE[r + 1] : x[r][c]);
        };
        auto D = [&](int r, int c) -> real { return X(r, c + 1) - X(r, c - 1); };
        // ---- boundary ring: rows 0 and BY-1 (all columns), then columns 0 and BX-1 ----
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int r = e == 0 ? 0 : BY - 1;
#pragma unroll
            for (int c = 0; c < BX; ++c)
                cell<J, SECOND>(out[r][c], x[r][c], X(r, c - 1), X(r + 1, c), X(r - 1, c), D(r, c),
                                D(r - 1, c), D(r + 1, c), aE[r][c], aN[r][c], k);
        }
#pragma unroll
        for (int r = 1; r < BY - 1; ++r)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int c = e == 0 ? 0 : BX - 1;
                cell<J, SECOND>(out[r][c], x[r][c], X(r, c - 1), X(r + 1, c), X(r - 1, c), D(r, c),
                                D(r - 1, c), D(r + 1, c), aE[r][c], aN[r][c], k);
            }
        publish_edges(sm, buf ^ 1, rank, tx, ty, out);
        asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    }

    // ---- row-paired kernel (SYNC = 4; one CTA per field, FP32) -------------
    // Rows r and r + BY/2 of a thread's block share one f32x2 register, so every
    // stencil operation is one FFMA2 / FADD2 for two cells: the same arithmetic
    // as stage() (a - b as fma(b, -1, a), which rounds like the subtraction) in
    // half the FP32 issue slots.  Pair row k holds rows (k, k + HB).
    static constexpr int HB = BY / 2;
    __device__ __forceinline__ static float2 psub(float2 a, float2 b)
    {
        return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
    }

    template <int J, bool SECOND>
    __device__ __forceinline__ static void stage_pair(real *sm, int buf, int tx, int ty,
                                                      const float2 (&x)[HB][BX], float2 (&out)[HB][BX],
                                                      const float2 (&aE)[HB][BX], const float2 (&aN)[HB][BX],
                                                      const CoefP &kp)
    {
        const int a0 = tx * BX, b0 = ty * BY;
        real *rowT = sm + buf * S::STAGE;
        real *rowB = rowT + S::ROW;
        real *colL = rowB + S::ROW;
        real *colR = colL + S::COL;
        {
            real t[BX], bt[BX];
#pragma unroll
            for (int c = 0; c < BX; ++c) { t[c] = x[0][c].x; bt[c] = x[HB - 1][c].y; }
            st_vec<real, BX>(rowT + ty * N + a0, t);
            st_vec<real, BX>(rowB + ty * N + a0, bt);
            real l[BY], r[BY];
#pragma unroll
            for (int q = 0; q < HB; ++q) {
                l[q] = x[q][0].x; l[q + HB] = x[q][0].y;
                r[q] = x[q][BX - 1].x; r[q + HB] = x[q][BX - 1].y;
            }
            st_vec<real, BY>(colL + tx * S::CS + b0, l);
            st_vec<real, BY>(colR + tx * S::CS + b0, r);
        }
        __syncthreads();
        real hS[BX], hN[BX], hW[BY + 2], hE[BY + 2];
        load_halos(sm, buf, tx, ty, hS, hN, hW, hE);
        // E-W differences: dm of pair row -1 = (south halo row, row HB-1), d0 of pair row 0
        float2 dm[BX], d0[BX], dp[BX];
#pragma unroll
        for (int c = 0; c < BX; ++c) {
            const float2 e = make_float2((c + 1 < BX) ? hS[c + 1] : hE[0],
                                         (c + 1 < BX) ? x[HB - 1][c + 1].x : hE[HB]);
            const float2 w = make_float2((c > 0) ? hS[c - 1] : hW[0],
                                         (c > 0) ? x[HB - 1][c - 1].x : hW[HB]);
            dm[c] = psub(e, w);
            const float2 e0 = (c + 1 < BX) ? x[0][c + 1] : make_float2(hE[1], hE[1 + HB]);
            const float2 w0 = (c > 0) ? x[0][c - 1] : make_float2(hW[1], hW[1 + HB]);
            d0[c] = psub(e0, w0);
        }
#pragma unroll
        for (int kr = 0; kr < HB; ++kr) {
#pragma unroll
            for (int c = 0; c < BX; ++c) {
                float2 e, w;
                if (kr + 1 < HB) {
                    e = (c + 1 < BX) ? x[kr + 1][c + 1] : make_float2(hE[kr + 2], hE[kr + 2 + HB]);
                    w = (c > 0) ? x[kr + 1][c - 1] : make_float2(hW[kr + 2], hW[kr + 2 + HB]);
                } else {                                // pair row HB = (row HB, north halo row)
                    e = make_float2((c + 1 < BX) ? x[0][c + 1].y : hE[HB + 1],
                                    (c + 1 < BX) ? hN[c + 1] : hE[BY + 1]);
                    w = make_float2((c > 0) ? x[0][c - 1].y : hW[HB + 1],
                                    (c > 0) ? hN[c - 1] : hW[BY + 1]);
                }
                dp[c] = psub(e, w);
            }
#pragma unroll
            for (int c = 0; c < BX; ++c) {
                const float2 xc = x[kr][c];
                const float2 xW = (c > 0) ? x[kr][c - 1] : make_float2(hW[kr + 1], hW[kr + 1 + HB]);
                const float2 xN = (kr + 1 < HB) ? x[kr + 1][c] : make_float2(x[0][c].y, hN[c]);
                const float2 xS = (kr > 0) ? x[kr - 1][c] : make_float2(hS[c], x[HB - 1][c].x);
                float2 d1 = d0[c], d2 = psub(xN, xS);
                if constexpr (J == 1) d1 = __fadd2_rn(d1, kp.T); else d2 = __fadd2_rn(d2, kp.T);
                const float2 cr = psub(dp[c], dm[c]);
                float2 g = __ffma2_rn(aE[kr][c], d1, SECOND ? out[kr][c] : kp.K);
                g = __ffma2_rn(kp.b11x2, xW, g);
                g = __ffma2_rn(aN[kr][c], d2, g);
                g = __ffma2_rn(kp.b22x2, xS, g);
                g = __ffma2_rn(kp.bx, cr, g);
                g = __ffma2_rn(kp.bc, xc, g);
                out[kr][c] = SECOND ? __ffma2_rn(g, make_float2(0.5f, 0.5f), kp.halfK) : g;
            }
#pragma unroll
            for (int c = 0; c < BX; ++c) { dm[c] = d0[c]; d0[c] = dp[c]; }
        }
    }

    // the time loop, flux sums and dump of the row-paired kernel
    template <int J>
    __device__ __forceinline__ static void pairs(const PatchParams &prm, real *sm, long long p, int tx,
                                                 int ty, const real (&A1)[BY][BX], const real (&A2)[BY][BX],
                                                 const Coef<real> &k, real b11, real b22, long long nb,
                                                 long long na, double &f1, double &f2)
    {
        static_assert(C == 1 && sizeof(real) == 4 && BY % 2 == 0, "row pairs: FP32, one CTA per field");
        float2 aE[HB][BX], aN[HB][BX], w[HB][BX], s[HB][BX];
#pragma unroll
        for (int q = 0; q < HB; ++q)
#pragma unroll
            for (int c = 0; c < BX; ++c) {
                aE[q][c] = make_float2(A1[q][c], A1[q + HB][c]);
                aN[q][c] = make_float2(A2[q][c], A2[q + HB][c]);
                w[q][c] = make_float2(0.f, 0.f);
            }
        CoefP kp;
        kp.b11x2 = make_float2(k.b11x2, k.b11x2);
        kp.b22x2 = make_float2(k.b22x2, k.b22x2);
        kp.bx = make_float2(k.bx, k.bx);
        kp.bc = make_float2(k.bc, k.bc);
        kp.T = make_float2(k.twoh, k.twoh);
        kp.K = make_float2(k.K, k.K);
        kp.halfK = make_float2(k.halfK, k.halfK);
        float2 p1 = make_float2(0.f, 0.f), p2 = p1, pw = p1;
        const double db11 = (double)b11, db22 = (double)b22;
        int win = 0;
        const long long ntot = nb + na;
        for (long long step = 0; step < ntot; ++step) {
            stage_pair<J, false>(sm, 0, tx, ty, w, s, aE, aN, kp);
            stage_pair<J, true>(sm, 1, tx, ty, s, w, aE, aN, kp);
            if (step >= nb) {
                float2 q1 = make_float2(0.f, 0.f), q2 = q1, qw = q1;
#pragma unroll
                for (int q = 0; q < HB; ++q)
#pragma unroll
                    for (int c = 0; c < BX; ++c) {
                        q1 = __ffma2_rn(aE[q][c], w[q][c], q1);
                        q2 = __ffma2_rn(aN[q][c], w[q][c], q2);
                        qw = __fadd2_rn(qw, w[q][c]);
                    }
                p1 = __fadd2_rn(p1, q1);
                p2 = __fadd2_rn(p2, q2);
                pw = __fadd2_rn(pw, qw);
                if (++win == kFlush) {
                    const double sw = (double)pw.x + (double)pw.y;
                    f1 += (double)p1.x + (double)p1.y - db11 * sw;
                    f2 += (double)p2.x + (double)p2.y - db22 * sw;
                    p1 = make_float2(0.f, 0.f); p2 = p1; pw = p1; win = 0;
                }
            }
        }
        const double sw = (double)pw.x + (double)pw.y;
        f1 += (double)p1.x + (double)p1.y - db11 * sw;
        f2 += (double)p2.x + (double)p2.y - db22 * sw;
        if (prm.wdump) {
            const int a0 = tx * BX, b0 = ty * BY;
            real *wd = static_cast<real *>(prm.wdump) + (2 * p + (J - 1)) * (long long)N * N;
#pragma unroll
            for (int q = 0; q < HB; ++q)
#pragma unroll
                for (int c = 0; c < BX; ++c) {
                    wd[(b0 + q) * N + a0 + c] = w[q][c].x;
                    wd[(b0 + q + HB) * N + a0 + c] = w[q][c].y;
                }
        }
    }

    // TM: the per-cell coefficients live in tensor memory at `tmem` (the CTA's
    // allocation of NT / 2 columns) instead of registers, see stage_tm(); TM = 2
    // reads the column halos as the rows need them.
    // GR: this field is one of several that groups of NT threads of the CTA
    // solve side by side (TM kernels, C = 1): `sm` is the group's own shared
    // memory, thread indices are group-local, barriers are the group's (csync).
    template <int J, int SYNC, int TM = 0, bool GR = false>
    __device__ static void run(const PatchParams &prm, real *sm, long long p, int rank,
                               uint32_t tmem = 0)
    {
        constexpr bool SPLIT = SYNC == 1;
        static_assert(TM == 0 || SYNC == 0 || SYNC == 3, "tensor-memory coefficients: SYNC 0 or 3");
        static_assert(!GR || (TM != 0 && C == 1 && SYNC == 0), "groups: TM kernels, one CTA per field");
        constexpr bool LZ = TM == 2;                    // column halos read as the rows need them
        const int tid = GR ? (int)(threadIdx.x % NT) : (int)threadIdx.x, tx = tid % NBX, ty = tid / NBX;
        const int a0 = tx * BX, b0 = ty * BY;          // slab-local
        const int g0 = rank * NS;                       // first patch row of the slab
        double *red = reinterpret_cast<double *>(sm + S::WORDS);
        // SYNC = 2: one mbarrier per stage buffer (slots 48, 49 of the reduction
        // area), 2 NBX arrivals per phase (NBX pushing threads in each neighbour);
        // the cluster barrier of the set-up orders the init before any arrival
        const uint32_t mbar0 = (uint32_t)__cvta_generic_to_shared(red + 48);
        if constexpr (SYNC == 2) {
            if (tid == 0) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mbar0), "r"(2 * NBX) : "memory");
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mbar0 + 8), "r"(2 * NBX) : "memory");
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            }
        }
        // SYNC = 3, 5: one arrival (thread 0's arm) and two incoming rows per phase;
        // the first phase of both barriers is armed here
        if constexpr (SYNC == 3 || SYNC == 5) {
            if (tid == 0) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbar0) : "memory");
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbar0 + 8) : "memory");
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
                arm_tx(mbar0, (uint32_t)(2 * N * sizeof(real)));
                arm_tx(mbar0 + 8, (uint32_t)(2 * N * sizeof(real)));
            }
        }
        const long long Nl = prm.Nl;
        const long long pi = p % prm.n_macro, pj = p / prm.n_macro;
        const long long ox = patch_origin(pi, prm.n_macro, Nl, N);
        const long long oy = patch_origin(pj, prm.n_macro, Nl, N);

        // ---- set-up: psi rows g0-1 .. g0+NS (patch-periodic), velocity, time step --
        real *psi = sm;
        const real *band = static_cast<const real *>(prm.band);
        for (int c = tid; c < N * (NS + 2); c += NT) {
            const int rr = c / N, a = c % N;
            const int b = (g0 - 1 + rr + N) % N;
            psi[c] = patch_band(band, Nl, prm.tile, p, ox, oy, N, a, b);
        }
        csync<GR>();
        const real inv2h = (real)(1.0 / (2.0 * prm.h));
        real A1[BY][BX], A2[BY][BX];
        real vmax = 0;
#pragma unroll
        for (int r = 0; r < BY; ++r) {
            const int rr = b0 + r + 1;                  // psi row of this cell
#pragma unroll
            for (int c = 0; c < BX; ++c) {
                const int a = a0 + c, ap = (a + 1) % N, am = (a + N - 1) % N;
                const real v1 = (psi[(rr - 1) * N + a] - psi[(rr + 1) * N + a]) * inv2h;
                const real v2 = (psi[rr * N + ap] - psi[rr * N + am]) * inv2h;
                A1[r][c] = v1;
                A2[r][c] = v2;
                vmax = fmax(vmax, fabs(v1) + fabs(v2));
            }
        }
        // patch max of |v1| + |v2|: warps -> CTA -> cluster (all ranks read all slots)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        if ((tid & 31) == 0) red[tid >> 5] = (double)vmax;
        csync<GR>();
        double vm = 0.0;
        for (int k = 0; k < NT / 32; ++k) vm = fmax(vm, red[k]);
        if constexpr (C > 1) {
            if (tid == 0) red[32] = vm;
            tile_sync<C>();
            vm = 0.0;
            for (int r = 0; r < C; ++r) vm = fmax(vm, *rank_ptr<C>(red + 32, r));
        }

        const double B11 = prm.Kb[3 * p], B12 = prm.Kb[3 * p + 1], B22 = prm.Kb[3 * p + 2];
        double dt;
        long long nb, na;
        micro_schedule(prm.h, prm.L, vm, B11, B12, B22, prm.cfl, prm.t_burn, prm.t_avg,
                       prm.nb_fixed, prm.na_fixed, dt, nb, na);
        // a base tensor that is not positive definite (or not finite) gives no usable
        // schedule: latch an error and return instead of stepping (every rank of the
        // cluster takes this branch together: same inputs, same arithmetic)
        if (!(dt > 0.0) || !isfinite(dt) || nb < 0 || na < 1 || nb + na > kMaxSteps) {
            if (tid == 0 && rank == 0) {
                prm.S[4 * p + 2 * (J - 1)] = __longlong_as_double(0x7ff8000000000000ll);
                prm.S[4 * p + 2 * (J - 1) + 1] = __longlong_as_double(0x7ff8000000000000ll);
                atomicCAS(prm.status, 0, MLSD_EINVAL);
            }
            if constexpr (C > 1) tile_sync<C>();   // no rank leaves while others read its slot
            return;
        }
        if (J == 1 && tid == 0 && rank == 0 && prm.steps) { prm.steps[p] = nb + na; prm.steps[prm.P + p] = na; }
        const double hh = prm.h * prm.h;
        const real cA = (real)(dt / (2.0 * prm.h));
        const real b11 = (real)(dt * B11 / hh), b22 = (real)(dt * B22 / hh);
        Coef<real> k;
        k.b11x2 = (real)2 * b11;
        k.b22x2 = (real)2 * b22;
        k.bx = (real)(dt * B12 / (2.0 * hh));
        k.bc = (real)(1.0 - 2.0 * (dt * B11 / hh + dt * B22 / hh));
        k.twoh = (real)(2.0 * prm.h);
        k.K = -k.twoh * (J == 1 ? b11 : b22);
        k.halfK = (real)0.5 * k.K;
        // A1, A2 become aE = A1 + b11, aN = A2 + b22 (A_i = dt v_i / 2h)
        const int warp = (int)(threadIdx.x >> 5);      // lane quarter and columns: CTA-wide warp
        const uint32_t tcol = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 64u * (uint32_t)(warp >> 2);
        if constexpr (TM) {
            // the same values, from v formed again from the psi rows, row by row into
            // tensor memory: (aE[0..3], aN[0..3]) of block row r at column 8 r
            __syncwarp();
#pragma unroll
            for (int r = 0; r < BY; ++r) {
                const int rr = b0 + r + 1;
                float cf[8];
#pragma unroll
                for (int c = 0; c < BX; ++c) {
                    const int a = a0 + c, ap = (a + 1) % N, am = (a + N - 1) % N;
                    const real v1 = (psi[(rr - 1) * N + a] - psi[(rr + 1) * N + a]) * inv2h;
                    const real v2 = (psi[rr * N + ap] - psi[rr * N + am]) * inv2h;
                    cf[c] = fma(v1, cA, b11);
                    cf[BX + c] = fma(v2, cA, b22);
                }
                tm_st8(tcol + 8 * r, cf);
            }
            tm_wait_st();
        } else {
#pragma unroll
            for (int r = 0; r < BY; ++r)
#pragma unroll
                for (int c = 0; c < BX; ++c) {
                    A1[r][c] = fma(A1[r][c], cA, b11);
                    A2[r][c] = fma(A2[r][c], cA, b22);
                }
        }
        // psi tile (and the vmax slots) are dead; the space becomes the exchange buffers
        if constexpr (C > 1) tile_sync<C>();
        else csync<GR>();

        double f1 = 0.0, f2 = 0.0;
        if constexpr (SYNC == 4) {
            pairs<J>(prm, sm, p, tx, ty, A1, A2, k, b11, b22, nb, na, f1, f2);
        } else {
        // ---- time stepping ------------------------------------------------
        real w[BY][BX], s[BY][BX];
#pragma unroll
        for (int r = 0; r < BY; ++r)
#pragma unroll
            for (int c = 0; c < BX; ++c) w[r][c] = 0;
        // flux sums: sum (A_i + b_ii) w = sum A_i w + b_ii sum w, so sum w is kept too
        real p1 = 0, p2 = 0, pw = 0;
        int win = 0;
        bool live = true;                               // SYNC = 2, 3: no wait has run out
        const long long ntot = nb + na;
        if constexpr (SPLIT) {
            publish_edges(sm, 0, rank, tx, ty, w);
            asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
        }
        for (long long step = 0; step < ntot; ++step) {
            if constexpr (TM) {
                const uint32_t par = (uint32_t)(step & 1);
                real q1 = 0, q2 = 0, qw = 0;
                stage_tm<J, false, SYNC, false, LZ, GR>(sm, 0, rank, tx, ty, w, s, tcol, k, mbar0,
                                                        par, prm.status, &live, q1, q2, qw);
                if (step < nb) {
                    stage_tm<J, true, SYNC, false, LZ, GR>(sm, 1, rank, tx, ty, s, w, tcol, k,
                                                           mbar0 + 8, par, prm.status, &live, q1, q2,
                                                           qw);
                    continue;
                }
                stage_tm<J, true, SYNC, true, LZ, GR>(sm, 1, rank, tx, ty, s, w, tcol, k, mbar0 + 8,
                                                      par, prm.status, &live, q1, q2, qw);
                p1 += q1;
                p2 += q2;
                pw += qw;
                if (++win == kFlush) {
                    f1 += (double)p1 - (double)b11 * (double)pw;
                    f2 += (double)p2 - (double)b22 * (double)pw;
                    p1 = 0; p2 = 0; pw = 0; win = 0;
                }
                continue;
            }
            if constexpr (SPLIT) {
                stage_split<J, false>(sm, 0, rank, tx, ty, w, s, A1, A2, k);
                stage_split<J, true>(sm, 1, rank, tx, ty, s, w, A1, A2, k);
            } else if constexpr (SYNC >= 2) {
                const uint32_t par = (uint32_t)(step & 1);
                stage<J, false, SYNC>(sm, 0, rank, tx, ty, w, s, A1, A2, k, mbar0, par, prm.status,
                                      &live);
                stage<J, true, SYNC>(sm, 1, rank, tx, ty, s, w, A1, A2, k, mbar0 + 8, par,
                                     prm.status, &live);
            } else {
                stage<J, false>(sm, 0, rank, tx, ty, w, s, A1, A2, k);
                stage<J, true>(sm, 1, rank, tx, ty, s, w, A1, A2, k);
            }
            if (step >= nb) {
                real q1 = 0, q2 = 0, qw = 0;
#pragma unroll
                for (int r = 0; r < BY; ++r)
#pragma unroll
                    for (int c = 0; c < BX; ++c) {
                        q1 = fma(A1[r][c], w[r][c], q1);
                        q2 = fma(A2[r][c], w[r][c], q2);
                        qw += w[r][c];
                    }
                p1 += q1;
                p2 += q2;
                pw += qw;
                if (++win == kFlush) {
                    f1 += (double)p1 - (double)b11 * (double)pw;
                    f2 += (double)p2 - (double)b22 * (double)pw;
                    p1 = 0; p2 = 0; pw = 0; win = 0;
                }
            }
        }
        f1 += (double)p1 - (double)b11 * (double)pw;
        f2 += (double)p2 - (double)b22 * (double)pw;
        if constexpr (SPLIT) asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");

        // ---- outputs ------------------------------------------------------
        if (prm.wdump) {
            real *wd = static_cast<real *>(prm.wdump) + (2 * p + (J - 1)) * (long long)N * N;
#pragma unroll
            for (int r = 0; r < BY; ++r)
#pragma unroll
                for (int c = 0; c < BX; ++c) wd[(g0 + b0 + r) * N + a0 + c] = w[r][c];
        }
        }   // SYNC != 4
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            f1 += __shfl_xor_sync(0xffffffffu, f1, o);
            f2 += __shfl_xor_sync(0xffffffffu, f2, o);
        }
        csync<GR>();
        if ((tid & 31) == 0) { red[2 * (tid >> 5)] = f1; red[2 * (tid >> 5) + 1] = f2; }
        csync<GR>();
        if (tid == 0) {
            double t1 = 0.0, t2 = 0.0;
            for (int k = 0; k < NT / 32; ++k) { t1 += red[2 * k]; t2 += red[2 * k + 1]; }
            red[40] = t1;
            red[41] = t2;
        }
        if constexpr (C > 1) tile_sync<C>();
        else csync<GR>();
        if (tid == 0 && rank == 0) {
            double t1 = 0.0, t2 = 0.0;
            for (int r = 0; r < C; ++r) { t1 += *rank_ptr<C>(red + 40, r); t2 += *rank_ptr<C>(red + 41, r); }
            // v_i = A_i / cA;  S_ij = (1/na) sum_steps mean_cells v_i w_j
            const double scale = 1.0 / ((double)cA * (double)N * (double)N * (double)na);
            const double s1j = t1 * scale, s2j = t2 * scale;
            prm.S[4 * p + 2 * (J - 1)] = s1j;
            prm.S[4 * p + 2 * (J - 1) + 1] = s2j;
            if (!isfinite(s1j) || !isfinite(s2j)) atomicCAS(prm.status, 0, MLSD_ENONFINITE);
        }
        if constexpr (C > 1) tile_sync<C>();   // keep every slab's shared memory alive until rank 0 has read it
    }
};

template <int N, int BX, int BY, typename real, int MINB, int C, int SYNC>
__global__ void __launch_bounds__((N / BX) * (N / C / BY), MINB)
k_patch_solve(PatchParams prm)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real *sm = reinterpret_cast<real *>(smem_raw);
    const int rank = (int)(blockIdx.x % C);
    if (!prm.count_dev) {
        // one work item per cluster (whole clusters only: C divides the grid)
        const long long item = prm.item0 + blockIdx.x / C;
        if (item >= prm.item0 + prm.items) return;
        const long long p = prm.pidx ? (long long)prm.pidx[item >> 1] : (item >> 1);
        if (item & 1) Tile<N, C, BX, BY, real>::template run<2, SYNC>(prm, sm, p, rank);
        else Tile<N, C, BX, BY, real>::template run<1, SYNC>(prm, sm, p, rank);
        return;
    }
    // a launch sized before the count was known: grid-stride loop over the first
    // 2 * (*count_dev) work items
    const long long end = prm.item0 + 2LL * (long long)*prm.count_dev;
    const long long stride = gridDim.x / C;
    for (long long item = prm.item0 + blockIdx.x / C; item < end; item += stride) {
        const long long p = prm.pidx ? (long long)prm.pidx[item >> 1] : (item >> 1);
        if (item & 1) Tile<N, C, BX, BY, real>::template run<2, SYNC>(prm, sm, p, rank);
        else Tile<N, C, BX, BY, real>::template run<1, SYNC>(prm, sm, p, rank);
    }
}

// Tilings with the per-cell coefficients in tensor memory (Tile::stage_tm): the
// CTA allocates NT / 2 TMEM columns once, runs its work items as k_patch_solve
// does, and frees them before it exits.
template <int N, int BX, int BY, int MINB, int C, int SYNC, int TM>
__global__ void __launch_bounds__((N / BX) * (N / C / BY), MINB)
k_patch_solve_tm(PatchParams prm)
{
    constexpr uint32_t COLS = (uint32_t)((N / BX) * (N / C / BY) / 2);
    static_assert(COLS >= 32 && (COLS & (COLS - 1)) == 0 && COLS <= 512, "TMEM allocation");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t tm_slot;
    float *sm = reinterpret_cast<float *>(smem_raw);
    const int rank = (int)(blockIdx.x % C);
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"((uint32_t)__cvta_generic_to_shared(&tm_slot)), "r"(COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tm_slot;
    using T = Tile<N, C, BX, BY, float>;
    // work items as in k_patch_solve: one per cluster, or a grid-stride walk over
    // the first 2 * (*count_dev) items when the launch was sized before the count
    const long long first = prm.item0 + blockIdx.x / C;
    const long long end = prm.count_dev ? prm.item0 + 2LL * (long long)*prm.count_dev
                                        : prm.item0 + prm.items;
    const long long stride = prm.count_dev ? (long long)(gridDim.x / C) : end;
    for (long long item = first; item < end; item += stride) {
        const long long p = prm.pidx ? (long long)prm.pidx[item >> 1] : (item >> 1);
        if (item & 1) T::template run<2, SYNC, TM>(prm, sm, p, rank, tmem);
        else T::template run<1, SYNC, TM>(prm, sm, p, rank, tmem);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(COLS)
                     : "memory");
    }
}

// SYNC: 0 = barrier per stage, 1 = split-phase cluster barrier, 2 = neighbour
// signalling, 3 = bulk copies of the slab edge rows, 5 = bulk copies with the
// cross-slab rows computed last (2, 3, 5: clusters only), 4 = row-paired
// f32x2 arithmetic (one CTA per field, FP32)
template <int N, int BX, int BY, typename real, int MINB = 1, int C = 1, int SYNC = 0>
void add_variant(std::vector<PatchVariant> &out)
{
    static_assert(SYNC < 2 || SYNC == 4 || C > 1, "neighbour signalling / bulk row copies need a cluster");
    static_assert(SYNC != 5 || BY >= 2, "deferred rows: two rows per block");
    static_assert(SYNC != 4 || (C == 1 && sizeof(real) == 4), "row pairs: FP32, one CTA per field");
    static_assert(((N / BX) * (N / C / BY)) % 32 == 0, "whole warps only");
    static_assert((N / BX) * (N / C / BY) <= 512, "reduction slots 0..31 (warp pairs), 32, 40, 41");
    static_assert(N % C == 0 && (N / C) % BY == 0 && N % BX == 0, "tiling");
    PatchVariant v;
    v.n = N;
    v.precision = sizeof(real) == 4 ? MLSD_FP32 : MLSD_FP64;
    v.bx = BX;
    v.by = BY;
    v.minb = MINB;
    v.packed = 0;
    v.cluster = C;
    v.split = SYNC;
    v.tmem = 0;
    v.threads = (N / BX) * (N / C / BY);
    v.smem = Smem<N, C, BX, BY, real>::BYTES;
    v.fn = reinterpret_cast<const void *>(&k_patch_solve<N, BX, BY, real, MINB, C, SYNC>);
    out.push_back(v);
}

// a tiling with the per-cell coefficients in tensor memory (FP32, 4 x 8 cells per
// thread); LZ: the column halos read as the rows need them
template <int N, int MINB = 1, int C = 1, int SYNC = 0, bool LZ = false>
void add_variant_tm(std::vector<PatchVariant> &out)
{
    constexpr int TM = LZ ? 2 : 1;
    constexpr int BX = 4, BY = 8;
    static_assert(((N / BX) * (N / C / BY)) % 128 == 0, "whole lane quarters of warps");
    static_assert((N / BX) * (N / C / BY) <= 512, "reduction slots 0..31 (warp pairs), 32, 40, 41");
    static_assert(N % C == 0 && (N / C) % BY == 0, "tiling");
    PatchVariant v;
    v.n = N;
    v.precision = MLSD_FP32;
    v.bx = BX;
    v.by = BY;
    v.minb = MINB;
    v.packed = 0;
    v.cluster = C;
    v.split = SYNC;
    v.tmem = TM;
    v.threads = (N / BX) * (N / C / BY);
    v.smem = Smem<N, C, BX, BY, float>::BYTES;
    v.fn = reinterpret_cast<const void *>(&k_patch_solve_tm<N, BX, BY, MINB, C, SYNC, TM>);
    out.push_back(v);
}

// ---------------------------------------------------------------------------
// Packed variant: one CTA advances BOTH corrector fields of a patch, each cell
// holding (w_1, w_2) in one float2 and every stencil operation issued as a
// Blackwell f32x2 instruction (FFMA2 / FADD2 / FMUL2).  The two fields share
// v, B and dt; only the source term differs, (2h, 0) on the E-W difference
// and (0, 2h) on the N-S difference.  a - b is formed as fma(b, -1, a), which
// rounds exactly like a subtraction, so the results equal the scalar kernel's.
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

template <int CNT>
__device__ __forceinline__ void st_vec2(float2 *dst, const float2 (&src)[CNT])
{
    static_assert(CNT % 2 == 0, "pairs of float2");
#pragma unroll
    for (int k = 0; k < CNT / 2; ++k)
        reinterpret_cast<float4 *>(dst)[k] =
            make_float4(src[2 * k].x, src[2 * k].y, src[2 * k + 1].x, src[2 * k + 1].y);
}

template <int CNT>
__device__ __forceinline__ void ld_vec2(float2 (&dst)[CNT], const float2 *src)
{
#pragma unroll
    for (int k = 0; k < CNT / 2; ++k) {
        const float4 v = reinterpret_cast<const float4 *>(src)[k];
        dst[2 * k] = make_float2(v.x, v.y);
        dst[2 * k + 1] = make_float2(v.z, v.w);
    }
}

template <int N, int BX, int BY>
struct Smem2 {
    static constexpr int NBX = N / BX, NBY = N / BY;
    static constexpr int CS = N + 2;              // column stride in float2 (16-byte pad)
    static constexpr int ROW = NBY * N, COL = NBX * CS;
    static constexpr int STAGE = 2 * ROW + 2 * COL;
    static constexpr int EXCH = 2 * STAGE;        // float2 words, double buffered
    static constexpr int SETUP = (N * N + 1) / 2; // psi tile (floats) in float2 words
    static constexpr int WORDS = (EXCH > SETUP ? EXCH : SETUP);
    static constexpr size_t BYTES = (size_t)WORDS * sizeof(float2) + 64 * sizeof(double);
};

template <int N, int BX, int BY>
struct Tile2 {
    static constexpr int NBX = N / BX, NBY = N / BY, NT = NBX * NBY;
    using S = Smem2<N, BX, BY>;

    template <bool SECOND>
    __device__ __forceinline__ static void stage(float2 *sm, int buf, int tx, int ty,
                                                 const float2 (&x)[BY][BX], float2 (&out)[BY][BX],
                                                 const float2 (&aE)[BY][BX], const float2 (&aN)[BY][BX],
                                                 float2 b11x2, float2 b22x2, float2 bx, float2 bc,
                                                 float2 T1, float2 T2, float2 K, float2 halfK)
    {
        const int a0 = tx * BX, b0 = ty * BY;
        float2 *rowT = sm + buf * S::STAGE;
        float2 *rowB = rowT + S::ROW;
        float2 *colL = rowB + S::ROW;
        float2 *colR = colL + S::COL;
        {
            float2 t[BX], bt[BX];
#pragma unroll
            for (int c = 0; c < BX; ++c) { t[c] = x[0][c]; bt[c] = x[BY - 1][c]; }
            st_vec2<BX>(rowT + ty * N + a0, t);
            st_vec2<BX>(rowB + ty * N + a0, bt);
            float2 l[BY], r[BY];
#pragma unroll
            for (int k = 0; k < BY; ++k) { l[k] = x[k][0]; r[k] = x[k][BX - 1]; }
            st_vec2<BY>(colL + tx * S::CS + b0, l);
            st_vec2<BY>(colR + tx * S::CS + b0, r);
        }
        __syncthreads();
        float2 hS[BX], hN[BX], hW[BY + 2], hE[BY + 2];
        {
            const int tyS = (ty + NBY - 1) % NBY, tyN = (ty + 1) % NBY;
            const int txW = (tx + NBX - 1) % NBX, txE = (tx + 1) % NBX;
            ld_vec2<BX>(hS, rowB + tyS * N + a0);
            ld_vec2<BX>(hN, rowT + tyN * N + a0);
            const float2 *cw = colR + txW * S::CS;
            const float2 *ce = colL + txE * S::CS;
            float2 tw[BY], te[BY];
            ld_vec2<BY>(tw, cw + b0);
            ld_vec2<BY>(te, ce + b0);
            const int bs = (b0 + N - 1) % N, bn = (b0 + BY) % N;
            hW[0] = cw[bs]; hE[0] = ce[bs];
            hW[BY + 1] = cw[bn]; hE[BY + 1] = ce[bn];
#pragma unroll
            for (int k = 0; k < BY; ++k) { hW[k + 1] = tw[k]; hE[k + 1] = te[k]; }
        }
        float2 dm[BX], d0[BX], dp[BX];
#pragma unroll
        for (int c = 0; c < BX; ++c) {
            const float2 e = (c + 1 < BX) ? hS[c + 1] : hE[0];
            const float2 w = (c > 0) ? hS[c - 1] : hW[0];
            dm[c] = sub2(e, w);
            const float2 e0 = (c + 1 < BX) ? x[0][c + 1] : hE[1];
            const float2 w0 = (c > 0) ? x[0][c - 1] : hW[1];
            d0[c] = sub2(e0, w0);
        }
#pragma unroll
        for (int r = 0; r < BY; ++r) {
#pragma unroll
            for (int c = 0; c < BX; ++c) {
                float2 e, w;
                if (r + 1 < BY) {
                    e = (c + 1 < BX) ? x[r + 1][c + 1] : hE[r + 2];
                    w = (c > 0) ? x[r + 1][c - 1] : hW[r + 2];
                } else {
                    e = (c + 1 < BX) ? hN[c + 1] : hE[BY + 1];
                    w = (c > 0) ? hN[c - 1] : hW[BY + 1];
                }
                dp[c] = sub2(e, w);
            }
#pragma unroll
            for (int c = 0; c < BX; ++c) {
                const float2 xc = x[r][c];
                const float2 xE = (c + 1 < BX) ? x[r][c + 1] : hE[r + 1];
                const float2 xW = (c > 0) ? x[r][c - 1] : hW[r + 1];
                const float2 xN = (r + 1 < BY) ? x[r + 1][c] : hN[c];
                const float2 xS = (r > 0) ? x[r - 1][c] : hS[c];
                (void)xE;
                // the scalar kernel's cell (Tile::cell) on both fields at once; the
                // sources differ per lane: T1 = (2h, 0), T2 = (0, 2h), K = -2h (b11, b22)
                const float2 d1 = __fadd2_rn(d0[c], T1);
                const float2 d2 = __fadd2_rn(sub2(xN, xS), T2);
                const float2 cr = sub2(dp[c], dm[c]);
                float2 g = __ffma2_rn(aE[r][c], d1, SECOND ? out[r][c] : K);
                g = __ffma2_rn(b11x2, xW, g);
                g = __ffma2_rn(aN[r][c], d2, g);
                g = __ffma2_rn(b22x2, xS, g);
                g = __ffma2_rn(bx, cr, g);
                g = __ffma2_rn(bc, xc, g);
                if constexpr (SECOND)
                    out[r][c] = __ffma2_rn(g, make_float2(0.5f, 0.5f), halfK);
                else
                    out[r][c] = g;
            }
#pragma unroll
            for (int c = 0; c < BX; ++c) { dm[c] = d0[c]; d0[c] = dp[c]; }
        }
    }

    __device__ static void run(const PatchParams &prm, float2 *sm, long long p)
    {
        const int tid = threadIdx.x, tx = tid % NBX, ty = tid / NBX;
        const int a0 = tx * BX, b0 = ty * BY;
        double *red = reinterpret_cast<double *>(sm + S::WORDS);
        const long long Nl = prm.Nl;
        const long long ox = patch_origin(p % prm.n_macro, prm.n_macro, Nl, N);
        const long long oy = patch_origin(p / prm.n_macro, prm.n_macro, Nl, N);
        float *psi = reinterpret_cast<float *>(sm);
        const float *band = static_cast<const float *>(prm.band);
        for (int c = tid; c < N * N; c += NT) {
            const int b = c / N, a = c % N;
            psi[c] = patch_band(band, Nl, prm.tile, p, ox, oy, N, a, b);
        }
        __syncthreads();
        const float inv2h = (float)(1.0 / (2.0 * prm.h));
        float v1r[BY][BX], v2r[BY][BX];
        float vmax = 0.f;
#pragma unroll
        for (int r = 0; r < BY; ++r) {
            const int b = b0 + r, bp = (b + 1) % N, bm = (b + N - 1) % N;
#pragma unroll
            for (int c = 0; c < BX; ++c) {
                const int a = a0 + c, ap = (a + 1) % N, am = (a + N - 1) % N;
                const float v1 = (psi[bm * N + a] - psi[bp * N + a]) * inv2h;
                const float v2 = (psi[b * N + ap] - psi[b * N + am]) * inv2h;
                v1r[r][c] = v1;
                v2r[r][c] = v2;
                vmax = fmaxf(vmax, fabsf(v1) + fabsf(v2));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        if ((tid & 31) == 0) red[tid >> 5] = (double)vmax;
        __syncthreads();
        double vm = 0.0;
        for (int k = 0; k < NT / 32; ++k) vm = fmax(vm, red[k]);

        const double B11 = prm.Kb[3 * p], B12 = prm.Kb[3 * p + 1], B22 = prm.Kb[3 * p + 2];
        double dt;
        long long nb, na;
        micro_schedule(prm.h, prm.L, vm, B11, B12, B22, prm.cfl, prm.t_burn, prm.t_avg,
                       prm.nb_fixed, prm.na_fixed, dt, nb, na);
        if (!(dt > 0.0) || !isfinite(dt) || nb < 0 || na < 1 || nb + na > kMaxSteps) {
            if (tid == 0) {
                const double qnan = __longlong_as_double(0x7ff8000000000000ll);
                for (int k = 0; k < 4; ++k) prm.S[4 * p + k] = qnan;
                atomicCAS(prm.status, 0, MLSD_EINVAL);
            }
            return;
        }
        if (tid == 0 && prm.steps) { prm.steps[p] = nb + na; prm.steps[prm.P + p] = na; }
        const double hh = prm.h * prm.h;
        const float cA = (float)(dt / (2.0 * prm.h));
        const float fb11 = (float)(dt * B11 / hh), fb22 = (float)(dt * B22 / hh);
        const float fbx = (float)(dt * B12 / (2.0 * hh));
        const float fbc = (float)(1.0 - 2.0 * (dt * B11 / hh + dt * B22 / hh));
        const float twoh = (float)(2.0 * prm.h);
        const float2 b11x2 = make_float2(2.f * fb11, 2.f * fb11), b22x2 = make_float2(2.f * fb22, 2.f * fb22);
        const float2 bx = make_float2(fbx, fbx), bc = make_float2(fbc, fbc);
        const float2 T1 = make_float2(twoh, 0.f), T2 = make_float2(0.f, twoh);
        const float2 K = make_float2(-twoh * fb11, -twoh * fb22);
        const float2 halfK = make_float2(0.5f * K.x, 0.5f * K.y);
        // aE = A1 + b11, aN = A2 + b22 with A_i = dt v_i / 2h
        float2 A1[BY][BX], A2[BY][BX];
#pragma unroll
        for (int r = 0; r < BY; ++r)
#pragma unroll
            for (int c = 0; c < BX; ++c) {
                const float a1 = fmaf(v1r[r][c], cA, fb11), a2 = fmaf(v2r[r][c], cA, fb22);
                A1[r][c] = make_float2(a1, a1);
                A2[r][c] = make_float2(a2, a2);
            }
        __syncthreads();

        float2 w[BY][BX], st[BY][BX];
#pragma unroll
        for (int r = 0; r < BY; ++r)
#pragma unroll
            for (int c = 0; c < BX; ++c) w[r][c] = make_float2(0.f, 0.f);
        // f_ij ~ sum A_i w_j = sum (A_i + b_ii) w_j - b_ii sum w_j
        float2 p1 = make_float2(0.f, 0.f), p2 = make_float2(0.f, 0.f), pw = make_float2(0.f, 0.f);
        double f11 = 0.0, f12 = 0.0, f21 = 0.0, f22 = 0.0;
        const double db11 = (double)fb11, db22 = (double)fb22;
        int win = 0;
        const long long ntot = nb + na;
        for (long long step = 0; step < ntot; ++step) {
            stage<false>(sm, 0, tx, ty, w, st, A1, A2, b11x2, b22x2, bx, bc, T1, T2, K, halfK);
            stage<true>(sm, 1, tx, ty, st, w, A1, A2, b11x2, b22x2, bx, bc, T1, T2, K, halfK);
            if (step >= nb) {
                float2 q1 = make_float2(0.f, 0.f), q2 = make_float2(0.f, 0.f), qw = make_float2(0.f, 0.f);
#pragma unroll
                for (int r = 0; r < BY; ++r)
#pragma unroll
                    for (int c = 0; c < BX; ++c) {
                        q1 = __ffma2_rn(A1[r][c], w[r][c], q1);
                        q2 = __ffma2_rn(A2[r][c], w[r][c], q2);
                        qw = __fadd2_rn(qw, w[r][c]);
                    }
                p1 = __fadd2_rn(p1, q1);
                p2 = __fadd2_rn(p2, q2);
                pw = __fadd2_rn(pw, qw);
                if (++win == kFlush) {
                    f11 += (double)p1.x - db11 * pw.x; f12 += (double)p1.y - db11 * pw.y;
                    f21 += (double)p2.x - db22 * pw.x; f22 += (double)p2.y - db22 * pw.y;
                    p1 = make_float2(0.f, 0.f); p2 = make_float2(0.f, 0.f); pw = make_float2(0.f, 0.f);
                    win = 0;
                }
            }
        }
        f11 += (double)p1.x - db11 * pw.x; f12 += (double)p1.y - db11 * pw.y;
        f21 += (double)p2.x - db22 * pw.x; f22 += (double)p2.y - db22 * pw.y;

        if (prm.wdump) {
            float *wd = static_cast<float *>(prm.wdump) + 2 * p * (long long)N * N;
#pragma unroll
            for (int r = 0; r < BY; ++r)
#pragma unroll
                for (int c = 0; c < BX; ++c) {
                    wd[(b0 + r) * N + a0 + c] = w[r][c].x;
                    wd[(long long)N * N + (b0 + r) * N + a0 + c] = w[r][c].y;
                }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            f11 += __shfl_xor_sync(0xffffffffu, f11, o);
            f12 += __shfl_xor_sync(0xffffffffu, f12, o);
            f21 += __shfl_xor_sync(0xffffffffu, f21, o);
            f22 += __shfl_xor_sync(0xffffffffu, f22, o);
        }
        __syncthreads();
        if ((tid & 31) == 0) {
            const int k = tid >> 5;
            red[4 * k] = f11; red[4 * k + 1] = f21; red[4 * k + 2] = f12; red[4 * k + 3] = f22;
        }
        __syncthreads();
        if (tid < 4) {
            double t = 0.0;
            for (int k = 0; k < NT / 32; ++k) t += red[4 * k + tid];
            // (S11, S21, S12, S22): v_i = A_i / cA, mean over cells and window
            const double v = t / ((double)cA * (double)N * (double)N * (double)na);
            prm.S[4 * p + tid] = v;
            if (!isfinite(v)) atomicCAS(prm.status, 0, MLSD_ENONFINITE);
        }
    }
};

template <int N, int BX, int BY, int MINB>
__global__ void __launch_bounds__((N / BX) * (N / BY), MINB)
k_patch_solve2(PatchParams prm)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    if (!prm.count_dev) {
        const long long pair = prm.item0 / 2 + blockIdx.x;
        if (2 * pair >= prm.item0 + prm.items) return;
        Tile2<N, BX, BY>::run(prm, sm, prm.pidx ? (long long)prm.pidx[pair] : pair);
        return;
    }
    const long long end = prm.item0 + 2LL * (long long)*prm.count_dev;
    for (long long pair = prm.item0 / 2 + blockIdx.x; 2 * pair < end; pair += gridDim.x)
        Tile2<N, BX, BY>::run(prm, sm, prm.pidx ? (long long)prm.pidx[pair] : pair);
}

template <int N, int BX, int BY, int MINB = 1>
void add_variant2(std::vector<PatchVariant> &out)
{
    static_assert(((N / BX) * (N / BY)) % 32 == 0, "whole warps only");
    static_assert((N / BX) * (N / BY) / 32 * 4 <= 64, "reduction scratch");
    PatchVariant v;
    v.n = N;
    v.precision = MLSD_FP32;
    v.bx = BX;
    v.by = BY;
    v.minb = MINB;
    v.packed = 1;
    v.cluster = 1;
    v.split = 0;
    v.tmem = 0;
    v.threads = (N / BX) * (N / BY);
    v.smem = Smem2<N, BX, BY>::BYTES;
    v.fn = reinterpret_cast<const void *>(&k_patch_solve2<N, BX, BY, MINB>);
    out.push_back(v);
}

}  // namespace
}  // namespace mlsd
