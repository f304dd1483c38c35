// Batched patch solve: the shared helpers and the failure-path check come from
// patch_kernels.cuh; the tilings are instantiated in patch_n32.cu, patch_n64.cu
// and patch_cluster.cu.  This unit holds the variant dispatch and the launches.
#include "patch_kernels.cuh"

namespace mlsd {
namespace {

// Failure-path check of nbr_wait (the cluster exchanges' bounded wait): one
// thread waits on a fresh mbarrier that receives no arrival and nothing else
// is in flight, so the wait expires and MLSD_ETIMEOUT is latched as in the
// patch kernels.
__global__ void k_wait_check_nbr(int *status)
{
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !nbr_wait(mb, 0, status)) atomicCAS(status, 0, MLSD_ETIMEOUT);
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" :: "r"(mb) : "memory");
}

__global__ void k_compose(long long P, const double *B, const double *S, double *K, int *status)
{
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const double *b = B + 3 * p, *s = S + 4 * p;
    // P_1 = B e_1 + S_.1, P_2 = B e_2 + S_.2; K = sym(P)
    double P11 = b[0] + s[0], P21 = b[1] + s[1], P12 = b[1] + s[2], P22 = b[2] + s[3];
    double k12 = 0.5 * (P21 + P12);
    K[3 * p] = P11;
    K[3 * p + 1] = k12;
    K[3 * p + 2] = P22;
    if (!isfinite(P11) || !isfinite(k12) || !isfinite(P22)) atomicCAS(status, 0, MLSD_ENONFINITE);
}

}  // namespace

cudaError_t launch_wait_check_nbr(int *status, cudaStream_t s)
{
    count_launches(1);
    k_wait_check_nbr<<<1, 32, 0, s>>>(status);
    return cudaGetLastError();
}

int patch_variants(int n, int precision, std::vector<PatchVariant> &out)
{
    // candidate thread-block tilings; the autotuner in the runtime times them
    out.clear();
    if (n == 32) return patch_variants_n32(precision, out);
    if (n == 64) return patch_variants_n64(precision, out);
    if ((n == 128 || n == 256) && precision == MLSD_FP32) return patch_variants_cluster(n, out);
    return 0;
}

cudaError_t launch_patch(const PatchVariant &v, const PatchParams &p, long long grid,
                         cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)v.smem);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<PatchParams *>(&p)};
    count_launches(1);
    if (v.cluster > 1 || v.split == 1) {        // barrier.cluster needs a cluster launch
        if (v.cluster > 8) {
            e = cudaFuncSetAttribute(v.fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(grid * v.cluster));
        cfg.blockDim = dim3(v.threads);
        cfg.dynamicSmemBytes = v.smem;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)v.cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelExC(&cfg, v.fn, args);
    }
    // packed kernels take one CTA per patch (both fields), item0 and grid even
    const long long g = v.packed ? (grid + 1) / 2 : grid;
    return cudaLaunchKernel(v.fn, dim3((unsigned)g), dim3(v.threads), args, v.smem, s);
}

cudaError_t launch_compose(long long P, const double *B, const double *S, double *K,
                           int *status, cudaStream_t s)
{
    const int t = 256;
    count_launches(1);
    k_compose<<<(unsigned)((P + t - 1) / t), t, 0, s>>>(P, B, S, K, status);
    return cudaGetLastError();
}

}  // namespace mlsd
