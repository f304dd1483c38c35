// One persistent launch for every patch of a level, whatever its size: the
// batched local solves of Sec. 2.2 (HMM steps 1-3) for a level whose patches
// have several grid sizes n in {32, 64, 128, 256} (Sec. 3's hierarchy with the
// resolution rule per patch).
//
// Every CTA has the same shape: 512 threads, the 4 x 8-cell blocks of the
// tensor-memory kernels (Tile::run with TM, the per-cell coefficients in the
// CTA's 256 TMEM columns), clusters of 4 CTAs.  A cluster takes one ticket at
// a time from the level's ticket list, static round-robin over the persistent
// clusters; a ticket is
//   * one 256^2 field: the 4 CTAs of the cluster hold its 4 row slabs of 64
//     rows and exchange their edge rows by bulk copies (SYNC 3), or
//   * four CTA tasks, one per CTA of the cluster: one 128^2 field (the whole
//     CTA), four 64^2 fields (groups of 128 threads on named barriers) or
//     sixteen 32^2 fields (one warp each).
// Each task is 65 536 cells.  The arithmetic of every field is that of the
// per-size kernels (Tile::run), so the results are the same bits.  The order of
// the tickets (the patch-to-CTA schedule) is built on the host and chosen by
// the runtime's trial of the level.
#include "patch_kernels.cuh"

namespace mlsd {
namespace {

constexpr int LV_THREADS = 512;
constexpr uint32_t LV_COLS = 256;

using T256 = Tile<256, 4, 4, 8, float>;
using T128 = Tile<128, 1, 4, 8, float>;
using T64 = Tile<64, 1, 4, 8, float>;
using T32 = Tile<32, 1, 4, 8, float>;
static_assert(T256::NT == LV_THREADS && T128::NT == LV_THREADS && T64::NT == 128 && T32::NT == 32,
              "task shapes");
static_assert(LevelParams::CLUSTER == 4 && T256::NS * LevelParams::CLUSTER == 256, "cluster of 4");

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t S256 = Smem<256, 4, 4, 8, float>::BYTES;
constexpr size_t S128 = Smem<128, 1, 4, 8, float>::BYTES;
constexpr size_t S64 = (Smem<64, 1, 4, 8, float>::BYTES + 15) / 16 * 16;
constexpr size_t S32 = (Smem<32, 1, 4, 8, float>::BYTES + 15) / 16 * 16;
constexpr size_t LV_SMEM = cmax(cmax(S256, S128), cmax(4 * S64, 16 * S32));

__device__ __forceinline__ long long patch_of(const PatchParams &pp, long long item)
{
    return pp.pidx ? (long long)pp.pidx[item >> 1] : (item >> 1);
}

__global__ void __launch_bounds__(LV_THREADS, 1) k_level_tm(const __grid_constant__ LevelParams lp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t tm_slot;
    const int rank = (int)(blockIdx.x % LevelParams::CLUSTER);
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"((uint32_t)__cvta_generic_to_shared(&tm_slot)), "r"(LV_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tm_slot;
    const long long clusters = gridDim.x / LevelParams::CLUSTER;
    for (long long t = blockIdx.x / LevelParams::CLUSTER; t < lp.n_tickets; t += clusters) {
        const long long code = lp.task[LevelParams::CLUSTER * t + rank];
        if (code >= 0) {
            const int sz = (int)(code >> 56);
            const long long item = code & ((1ll << 56) - 1);
            const PatchParams &pp = lp.cls[sz];
            float *sm = reinterpret_cast<float *>(smem_raw);
            if (sz == 3) {                        // one 256^2 field over the cluster
                const long long p = patch_of(pp, item);
                if (item & 1) T256::run<2, 3, 2>(pp, sm, p, rank, tmem);
                else T256::run<1, 3, 2>(pp, sm, p, rank, tmem);
                if (threadIdx.x == 0) {
                    // its two exchange mbarriers: the memory is reused by the next task
                    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(
                        reinterpret_cast<double *>(sm + Smem<256, 4, 4, 8, float>::WORDS) + 48);
                    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" :: "r"(mb) : "memory");
                    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" :: "r"(mb + 8) : "memory");
                }
            } else if (sz == 2) {                 // one 128^2 field per CTA
                const long long p = patch_of(pp, item);
                if (item & 1) T128::run<2, 0, 2>(pp, sm, p, 0, tmem);
                else T128::run<1, 0, 2>(pp, sm, p, 0, tmem);
            } else if (sz == 1) {                 // four 64^2 fields, 128 threads each
                const int g = (int)(threadIdx.x / 128);
                const long long it = item + g;
                if (it < pp.items) {
                    float *gs = reinterpret_cast<float *>(smem_raw + g * S64);
                    const long long p = patch_of(pp, it);
                    if (it & 1) T64::run<2, 0, 2, true>(pp, gs, p, 0, tmem);
                    else T64::run<1, 0, 2, true>(pp, gs, p, 0, tmem);
                }
            } else {                              // sixteen 32^2 fields, one warp each
                const int g = (int)(threadIdx.x / 32);
                const long long it = item + g;
                if (it < pp.items) {
                    float *gs = reinterpret_cast<float *>(smem_raw + g * S32);
                    const long long p = patch_of(pp, it);
                    if (it & 1) T32::run<2, 0, 2, true>(pp, gs, p, 0, tmem);
                    else T32::run<1, 0, 2, true>(pp, gs, p, 0, tmem);
                }
            }
        }
        // the next task may use other threads' shared memory and TMEM columns
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(LV_COLS)
                     : "memory");
    }
}

}  // namespace

size_t level_kernel_smem() { return LV_SMEM; }

// Resident clusters of the level kernel on this device (at least 1 when it fits at all).
cudaError_t level_kernel_clusters(int *out)
{
    *out = 0;
    const void *fn = reinterpret_cast<const void *>(&k_level_tm);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LV_SMEM);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(LevelParams::CLUSTER);
    cfg.blockDim = dim3(LV_THREADS);
    cfg.dynamicSmemBytes = LV_SMEM;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = LevelParams::CLUSTER;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(out, fn, &cfg);
}

cudaError_t launch_level(const LevelParams &lp, int clusters, cudaStream_t s)
{
    const void *fn = reinterpret_cast<const void *>(&k_level_tm);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LV_SMEM);
    if (e != cudaSuccess) return e;
    const long long g = std::min<long long>(clusters, lp.n_tickets);
    if (g < 1) return cudaSuccess;
    count_launches(1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(g * LevelParams::CLUSTER));
    cfg.blockDim = dim3(LV_THREADS);
    cfg.dynamicSmemBytes = LV_SMEM;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = LevelParams::CLUSTER;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    void *args[] = {const_cast<LevelParams *>(&lp)};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace mlsd
