// Tensor-core (tcgen05) inference of the surrogate ensemble: one CTA runs all
// four layers of one member on a 128-row tile.
//
//   * operands are staged in shared memory in the canonical no-swizzle
//     K-major layout: 8-row x 16-byte core matrices, consecutive along K
//     (leading-byte offset 128 B) and SBO bytes apart along M / N;
//   * one elected thread issues tcgen05.mma (kind::f16, bfloat16 A and B,
//     FP32 accumulator in tensor memory, M = 128, K = 16 per instruction),
//     tcgen05.commit signals an mbarrier the CTA waits on (bounded);
//   * the epilogue reads the accumulator rows with tcgen05.ld (thread t of
//     warp w owns row 32 w + t), adds the bias, applies the exact-erf GELU,
//     rounds to bfloat16 and writes the next layer's A operand in shared memory.
// A wait that exceeds its iteration limit latches MLSD_ETIMEOUT, skips the rest
// of the tile, frees the tensor memory and returns.
#include <cuda_bf16.h>

#include <cstdint>

#include "mlsd_internal.cuh"

namespace mlsd {
namespace {

constexpr int TM = 128;                // rows per tile (MMA M)
constexpr int KC = 64;                 // K chunk staged per round
constexpr int HMAX = 256;              // hidden width supported by this kernel
constexpr unsigned TMEM_COLS = 256;
constexpr long long kWaitLimit = 1ll << 24;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// no-swizzle K-major shared-memory matrix descriptor (sm_100 family)
__device__ __forceinline__ uint64_t mat_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;              // descriptor version for tcgen05
    return d;                            // base offset 0, swizzle none
}

// instruction descriptor: D FP32, A and B bfloat16, both K-major, M x N
__host__ __device__ constexpr uint32_t inst_desc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(mbar) : "memory");
}

// bounded wait for the mbarrier phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (long long it = 0; it < kWaitLimit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float gelu_tc(float z)
{
    return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}

// byte offset of element (r, k) in a no-swizzle K-major tile with K columns
__device__ __forceinline__ uint32_t cm_off(int r, int k, int K)
{
    return (uint32_t)(((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// stage rows [0, R) x columns [k0, k0 + KC) of a row-major bfloat16 matrix (ld elements
// per row, rows >= rows_valid read as zero) into a core-matrix tile with K = KC
__device__ __forceinline__ void stage_chunk(unsigned char *dst, const __nv_bfloat16 *src, int R,
                                            int rows_valid, long long ld, int k0)
{
    for (int t = threadIdx.x; t < R * (KC / 8); t += blockDim.x) {
        const int r = t / (KC / 8), kc = t % (KC / 8);
        uint4 v = make_uint4(0, 0, 0, 0);
        if (r < rows_valid) v = *reinterpret_cast<const uint4 *>(src + (long long)r * ld + k0 + 8 * kc);
        *reinterpret_cast<uint4 *>(dst + cm_off(r, 8 * kc, KC)) = v;
    }
}

struct TcArgs {
    const __nv_bfloat16 *X;      // [M][640]
    long long M;
    int h, members;
    const __nv_bfloat16 *const *wb;   // per member bfloat16 parameters (layout of the ABI)
    const float *const *wf;           // per member FP32 parameters (biases are read here)
    float *out;                  // [members][M][3]
    int *status;
};

__global__ void __launch_bounds__(128, 1) k_mlp_tc(TcArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *As = smem;                        // [128][64] bf16 chunk, 16 KB
    unsigned char *Bs = As + TM * KC * 2;            // [256][64] bf16 chunk, 32 KB
    unsigned char *Hs = Bs + HMAX * KC * 2;          // [128][256] bf16 activations, 64 KB
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;

    const int member = blockIdx.y;
    const long long row0 = (long long)blockIdx.x * TM;
    const int rows_valid = (int)min((long long)TM, a.M - row0);
    const int h = a.h;
    const __nv_bfloat16 *wb = a.wb[member];
    const float *wf = a.wf[member];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // parameter offsets (W1 b1 W2 b2 W3 b3 W4 b4)
    const long long oW1 = 0, ob1 = oW1 + (long long)h * MLSD_SUR_IN, oW2 = ob1 + h;
    const long long ob2 = oW2 + (long long)h * h, oW3 = ob2 + h, ob3 = oW3 + (long long)h * h;
    const long long oW4 = ob3 + h, ob4 = oW4 + 3LL * h;

    if (threadIdx.x == 0) {
        failed = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_slot)), "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t mb = smem_u32(&mbar);
    uint32_t phase = 0;
    const uint32_t taddr_row = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's 32 lanes

    // one layer: D[128][N] = A[128][K] W^T with W [N][K] row-major in global memory.
    // a_from_h: A is the activation tile in Hs (K = h), else X chunks from global.
    auto layer = [&](bool a_from_h, int K, int N, int n_rows_w, const __nv_bfloat16 *W) -> bool {
        const uint32_t idesc = inst_desc(TM, N);
        for (int k0 = 0; k0 < K; k0 += KC) {
            if (!a_from_h) stage_chunk(As, a.X + row0 * MLSD_SUR_IN, TM, rows_valid, MLSD_SUR_IN, k0);
            stage_chunk(Bs, W, N, n_rows_w, K, k0);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (threadIdx.x == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int ks = 0; ks < KC / 16; ++ks) {
                    uint64_t da, db;
                    if (a_from_h) da = mat_desc(smem_u32(Hs + ((k0 + ks * 16) >> 3) * 128), 128, (h >> 3) * 128);
                    else da = mat_desc(smem_u32(As + ks * 2 * 128), 128, (KC >> 3) * 128);
                    db = mat_desc(smem_u32(Bs + ks * 2 * 128), 128, (KC >> 3) * 128);
                    mma_bf16(tmem, da, db, idesc, (k0 > 0 || ks > 0) ? 1u : 0u);
                }
                mma_commit(mb);
            }
            const bool ok = mbar_wait(mb, phase);
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!ok) { failed = 1; }
            __syncthreads();
            if (failed) return false;
        }
        return true;
    };

    // epilogue: bias + GELU -> bfloat16 activations in Hs (K = h)
    auto epilogue_hidden = [&](const float *bias) {
        const int r = warp * 32 + lane;
        for (int c0 = 0; c0 < h; c0 += 16) {
            float v[16];
            tmem_ld16(taddr_row + (uint32_t)c0, v);
            __align__(16) __nv_bfloat16 o[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) o[i] = __float2bfloat16_rn(gelu_tc(v[i] + bias[c0 + i]));
            *reinterpret_cast<uint4 *>(Hs + cm_off(r, c0, h)) = *reinterpret_cast<const uint4 *>(o);
            *reinterpret_cast<uint4 *>(Hs + cm_off(r, c0 + 8, h)) = *reinterpret_cast<const uint4 *>(o + 8);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    };

    bool ok = layer(false, MLSD_SUR_IN, h, h, wb + oW1);
    if (ok) { epilogue_hidden(wf + ob1); ok = layer(true, h, h, h, wb + oW2); }
    if (ok) { epilogue_hidden(wf + ob2); ok = layer(true, h, h, h, wb + oW3); }
    if (ok) { epilogue_hidden(wf + ob3); ok = layer(true, h, 16, 3, wb + oW4); }
    if (ok) {
        const int r = warp * 32 + lane;
        float v[16];
        tmem_ld16(taddr_row, v);
        if (r < rows_valid) {
            float *o = a.out + ((long long)member * a.M + row0 + r) * 3;
            o[0] = v[0] + wf[ob4];
            o[1] = v[1] + wf[ob4 + 1];
            o[2] = v[2] + wf[ob4 + 2];
        }
    } else if (threadIdx.x == 0) {
        atomicCAS(a.status, 0, MLSD_ETIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS));
    }
}

}  // namespace

size_t mlp_tc_smem() { return (size_t)TM * KC * 2 + (size_t)HMAX * KC * 2 + (size_t)TM * HMAX * 2; }

bool mlp_tc_supported(int h) { return h % 64 == 0 && h <= HMAX && h >= 64; }

cudaError_t launch_mlp_tc(const void *X, long long M, int h, int members, const void *const *wb_dev,
                          const float *const *wf_dev, float *out, int *status, cudaStream_t s)
{
    TcArgs a;
    a.X = static_cast<const __nv_bfloat16 *>(X);
    a.M = M;
    a.h = h;
    a.members = members;
    a.wb = reinterpret_cast<const __nv_bfloat16 *const *>(wb_dev);
    a.wf = wf_dev;
    a.out = out;
    a.status = status;
    const size_t smem = mlp_tc_smem();
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(&k_mlp_tc),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((M + TM - 1) / TM), (unsigned)members);
    count_launches(1);
    k_mlp_tc<<<grid, 128, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mlsd
