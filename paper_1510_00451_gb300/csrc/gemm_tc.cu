// Tensor-core (tcgen05) GEMMs of the surrogate's training step:
//   D[M][N] = A[M][K] B[N][K]^T, A and B bfloat16 with K contiguous (K-major),
//   FP32 accumulation in tensor memory, one 128 x BN output tile per CTA and
//   optionally one slice of K per CTA (gridDim.z slices, partial sums).
// Operands arrive by cp.async.bulk.tensor through 3-D core-matrix views into a
// ring of mbarrier-guarded slots (6 of 32 KB, or 4 of 48 KB for 256-column tiles); one thread issues the MMAs
// (kind::f16, M = 128, N = BN, K = 16 per instruction) and commits each slot's
// release and the accumulator; the epilogue reads the accumulator rows with
// tcgen05.ld (warp w owns the TMEM lanes of quarter w % 4).  Epilogues:
//   forward  Z = D + bias (FP32), act = bf16(gelu(Z)) and its transpose;
//   backward dZ = bf16(D gelu'(Zprev)) and its transpose (the rounding of the
//            hidden layers' gradients to bfloat16 operands);
//   partial  the raw FP32 D of the CTA's K slice.
// Transposed outputs have rows ldT elements apart; entries m in [M, ldT) are
// written as zeros, so the padding a later view reads past K = M is zero.
// A wait that runs out latches MLSD_ETIMEOUT, lets the copies in flight land
// (bounded), frees the tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>

#include "mlsd_internal.cuh"

namespace mlsd {
namespace {

constexpr int GT_M = 128;                  // rows per tile (MMA M)
constexpr int GT_KC = 64;                  // K elements per ring slot
// ring slots per tile width: 192 KB of shared memory either way
template <int BN> constexpr int gt_ring() { return BN == 64 ? 8 : (BN == 128 ? 6 : 4); }
constexpr int GT_THREADS = 256;            // 8 warps
constexpr long long kGtWaitClocks = 1ll << 31;

enum { GT_FWD = 0, GT_BWD = 1, GT_PART = 2 };

struct GtArgs {
    CUtensorMap amap, bmap;                // A [M][K] (box 128 rows), B [N][K] (box BN rows)
    int M, N, K, kc_slice;                 // kc_slice: K chunks of GT_KC per CTA slice
    int mode;
    const float *bias;                     // forward
    float *Z;                              // forward: [M][N]
    const float *Zprev;                    // backward: [M][N]
    __nv_bfloat16 *out, *outT;             // forward act / backward dZ: [M][N] and [N][ldT]
    int ldT;
    float *part;                           // partial: [gridDim.z][M][N]
    int *status;
};

__device__ __forceinline__ uint32_t s_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// no-swizzle K-major shared-memory matrix descriptor (tcgen05 version bit set)
__device__ __forceinline__ uint64_t gt_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor: D FP32, A and B bfloat16, both K-major, M x N
__device__ __forceinline__ uint32_t gt_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool gt_wait(uint32_t mbar, uint32_t parity)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
        if (ok) return true;
        if (clock64() - t0 > kGtWaitClocks) return false;
    }
}

__device__ __forceinline__ void gt_tma3(uint32_t dst, const CUtensorMap *map, int c1, int c2,
                                        uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(c1), "r"(c2), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ float gt_gelu(float z)
{
    return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gt_gelu_d(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

template <int BN>
__global__ void __launch_bounds__(GT_THREADS, 1) k_gemm_tc(const __grid_constant__ GtArgs a)
{
    constexpr int A_BYTES = GT_M * GT_KC * 2, B_BYTES = BN * GT_KC * 2, SLOT = A_BYTES + B_BYTES;
    constexpr int GT_RING = gt_ring<BN>();
    constexpr uint32_t TCOLS = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[GT_RING], empty[GT_RING], accb;
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * GT_M, n0 = blockIdx.x * BN;
    const int kc_total = (a.K + GT_KC - 1) / GT_KC;
    const int kc0 = blockIdx.z * a.kc_slice;
    const int nk = max(0, min(a.kc_slice, kc_total - kc0));
    const CUtensorMap *pa = &a.amap, *pb = &a.bmap;

    if (threadIdx.x == 0) {
        failed = 0;
        for (int i = 0; i < GT_RING; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(s_u32(&full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(s_u32(&empty[i])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(s_u32(&accb)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(s_u32(&tmem_slot)), "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    auto issue = [&](int q) {
        const int slot = q % GT_RING;
        unsigned char *sA = smem + slot * SLOT, *sB = sA + A_BYTES;
        const uint32_t fb = s_u32(&full[slot]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     :: "r"(fb), "r"((uint32_t)SLOT) : "memory");
        const int kg = (kc0 + q) * (GT_KC / 8);
        gt_tma3(s_u32(sA), pa, m0, kg, fb);
        gt_tma3(s_u32(sB), pb, n0, kg, fb);
    };

    bool ok = true;
    int issued = 0, q = 0;
    if (threadIdx.x == 0 && nk > 0) {
        for (; issued < GT_RING && issued < nk; ++issued) issue(issued);
        const uint32_t idesc = gt_idesc(GT_M, BN);
        for (; q < nk; ++q) {
            const int slot = q % GT_RING;
            if (!gt_wait(s_u32(&full[slot]), (uint32_t)((q / GT_RING) & 1))) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            unsigned char *sA = smem + slot * SLOT, *sB = sA + A_BYTES;
#pragma unroll
            for (int ks = 0; ks < GT_KC / 16; ++ks) {
                const uint64_t da = gt_desc(s_u32(sA + ks * 2 * (GT_M * 16)), GT_M * 16, 128);
                const uint64_t db = gt_desc(s_u32(sB + ks * 2 * (BN * 16)), BN * 16, 128);
                const uint32_t acc = (q > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.u32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                    :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(s_u32(&empty[slot])) : "memory");
            // refill the slot of the previous chunk once its MMAs are done
            const int qn = q - 1 + GT_RING;
            if (q >= 1 && qn < nk) {
                const int ps = (q - 1) % GT_RING;
                if (!gt_wait(s_u32(&empty[ps]), (uint32_t)(((q - 1) / GT_RING) & 1))) { ok = false; break; }
                issue(qn);
                issued = qn + 1;
            }
        }
        if (ok)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(s_u32(&accb)) : "memory");
        else
            failed = 1;
    }
    __syncthreads();
    if (nk > 0 && !failed) {
        const bool got = gt_wait(s_u32(&accb), 0);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!got) failed = 1;
    }
    __syncthreads();
    if (!failed) {
        // epilogue: warp w reads rows 32 (w % 4) + lane and the 32-column chunks
        // (w / 4), (w / 4) + 2, ... of the tile
        const int lq = warp & 3, cg = warp >> 2;
        const int r = lq * 32 + lane, m = m0 + r;
        const uint32_t trow = tmem + ((uint32_t)(lq * 32) << 16);
        for (int c0 = 32 * cg; c0 < BN; c0 += 32 * (GT_THREADS / 128)) {
            if (n0 + c0 >= a.N) break;
            float v[32];
            if (nk > 0) {
                uint32_t rr[32];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
                    "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]),
                      "=r"(rr[6]), "=r"(rr[7]), "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]),
                      "=r"(rr[12]), "=r"(rr[13]), "=r"(rr[14]), "=r"(rr[15]), "=r"(rr[16]),
                      "=r"(rr[17]), "=r"(rr[18]), "=r"(rr[19]), "=r"(rr[20]), "=r"(rr[21]),
                      "=r"(rr[22]), "=r"(rr[23]), "=r"(rr[24]), "=r"(rr[25]), "=r"(rr[26]),
                      "=r"(rr[27]), "=r"(rr[28]), "=r"(rr[29]), "=r"(rr[30]), "=r"(rr[31])
                    : "r"(trow + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(rr[i]);
            } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.f;
            }
            // N is a multiple of 32 and so is n0 + c0: the whole chunk is inside the matrix
            const int nb = n0 + c0;
            if (a.mode == GT_PART) {
                if (m < a.M) {
                    float *dst = a.part + ((long long)blockIdx.z * a.M + m) * a.N + nb;
#pragma unroll
                    for (int i = 0; i < 32; i += 4)
                        *reinterpret_cast<float4 *>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                }
                continue;
            }
            // the thread's row segment of 32 columns moves as 16-byte vectors; the
            // transposed output is written column by column (consecutive lanes,
            // consecutive rows: one 64-byte segment per column)
            __align__(16) __nv_bfloat16 o[32];
            if (m < a.M) {
                const long long e0 = (long long)m * a.N + nb;
                if (a.mode == GT_FWD) {
#pragma unroll
                    for (int i = 0; i < 32; i += 4) {
                        const float4 b = *reinterpret_cast<const float4 *>(a.bias + nb + i);
                        const float4 z = make_float4(v[i] + b.x, v[i + 1] + b.y, v[i + 2] + b.z, v[i + 3] + b.w);
                        if (a.Z) *reinterpret_cast<float4 *>(a.Z + e0 + i) = z;
                        o[i] = __float2bfloat16_rn(gt_gelu(z.x));
                        o[i + 1] = __float2bfloat16_rn(gt_gelu(z.y));
                        o[i + 2] = __float2bfloat16_rn(gt_gelu(z.z));
                        o[i + 3] = __float2bfloat16_rn(gt_gelu(z.w));
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 32; i += 4) {
                        const float4 zp = *reinterpret_cast<const float4 *>(a.Zprev + e0 + i);
                        o[i] = __float2bfloat16_rn(v[i] * gt_gelu_d(zp.x));
                        o[i + 1] = __float2bfloat16_rn(v[i + 1] * gt_gelu_d(zp.y));
                        o[i + 2] = __float2bfloat16_rn(v[i + 2] * gt_gelu_d(zp.z));
                        o[i + 3] = __float2bfloat16_rn(v[i + 3] * gt_gelu_d(zp.w));
                    }
                }
#pragma unroll
                for (int i = 0; i < 32; i += 8)
                    *reinterpret_cast<uint4 *>(a.out + e0 + i) = *reinterpret_cast<const uint4 *>(o + i);
            } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) o[i] = __float2bfloat16_rn(0.f);
            }
            if (a.outT && m < a.ldT) {
#pragma unroll
                for (int i = 0; i < 32; ++i) a.outT[(long long)(nb + i) * a.ldT + m] = o[i];
            }
        }
    }
    if (failed && threadIdx.x == 0) {
        atomicCAS(a.status, 0, MLSD_ETIMEOUT);
        // let the copies still in flight land (bounded) before the CTA leaves
        for (int k = q; k < issued; ++k) gt_wait(s_u32(&full[k % GT_RING]), (uint32_t)((k / GT_RING) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TCOLS));
    }
}

template <int BN>
cudaError_t launch_gt(const GtArgs &a, int splits, cudaStream_t s)
{
    constexpr size_t smem = (size_t)gt_ring<BN>() * (GT_M * GT_KC * 2 + BN * GT_KC * 2);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(&k_gemm_tc<BN>),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 g((unsigned)((a.N + BN - 1) / BN), (unsigned)((a.M + GT_M - 1) / GT_M), (unsigned)splits);
    count_launches(1);
    k_gemm_tc<BN><<<g, GT_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

// One tensor-core GEMM (see the top of the file).  A: M rows of K bfloat16
// elements, lda apart; B: N rows of K, ldb apart (lda, ldb multiples of 8, both at
// least K rounded up to 8, their padding zero).  mode 0 forward (bias, Z, act,
// actT), 1 backward (Zprev, dZ, dZT), 2 partial sums of up to `splits` K slices
// into part [slices][M][N], the number of slices used returned in *slices.  In the
// forward mode Z and the transpose may be NULL.
// BN = 128, or 64 where 128-column tiles would fill less than a third of the SMs
// (256 with MLSD_GEMM_BN=256 where N is a multiple of 256).
cudaError_t gemm_tc(int mode, int M, int N, int K, const void *A, long long lda, const void *B,
                    long long ldb, const float *bias, float *Z, const float *Zprev, void *out,
                    void *outT, int ldT, float *part, int splits, int *slices, int *status,
                    cudaStream_t s)
{
    if (M < 1 || N < 1 || K < 1 || splits < 1 || N % 32) return cudaErrorInvalidValue;
    if (mode != GT_PART) splits = 1;
    // 128-column tiles: twice the CTAs of 256-column ones on these short GEMMs
    // (MLSD_GEMM_BN=256 selects the wide tile where N is a multiple of 256)
    static const bool wide = [] { const char *e = std::getenv("MLSD_GEMM_BN"); return e && std::atoi(e) == 256; }();
    // 64-column tiles where 128-column ones would leave most SMs idle
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 152;
    const long long tiles128 = (long long)((N + 127) / 128) * ((M + GT_M - 1) / GT_M) * splits;
    const int bn = (wide && N % 256 == 0) ? 256 : (tiles128 * 3 < sms ? 64 : 128);
    GtArgs a;
    if (!encode_rows_bf16(&a.amap, A, M, K, lda, GT_M) ||
        !encode_rows_bf16(&a.bmap, B, N, K, ldb, bn))
        return cudaErrorNotSupported;
    a.M = M; a.N = N; a.K = K;
    const int kc_total = (K + GT_KC - 1) / GT_KC;
    splits = std::min(splits, kc_total);
    a.kc_slice = (kc_total + splits - 1) / splits;
    splits = (kc_total + a.kc_slice - 1) / a.kc_slice;       // no empty slice
    a.mode = mode;
    a.bias = bias; a.Z = Z; a.Zprev = Zprev;
    a.out = static_cast<__nv_bfloat16 *>(out);
    a.outT = static_cast<__nv_bfloat16 *>(outT);
    a.ldT = ldT;
    a.part = part;
    a.status = status;
    if (slices) *slices = splits;
    return bn == 256 ? launch_gt<256>(a, splits, s)
                     : (bn == 128 ? launch_gt<128>(a, splits, s) : launch_gt<64>(a, splits, s));
}

int gemm_tc_splits(int M, int N, int K, int sms)
{
    // enough K slices that the tiles fill the GPU, each at least 4 chunks deep
    const int tiles = ((N + 127) / 128) * ((M + GT_M - 1) / GT_M);
    const int kc = (K + GT_KC - 1) / GT_KC;
    return std::max(1, std::min(kc / 4, sms / std::max(1, tiles)));
}

}  // namespace mlsd
