// dg_cdft_mma.cu -- the chunked-DFT contraction on the 5th-generation tensor
// cores (tcgen05, sm_103a), 16-bit products accumulated in FP32.
//
// For one snapshot the contraction is one tall GEMM. Its rows are the
// (lag bucket, chunk) pairs (NB x B rows). For chunk b of lag L the row holds
// the lag products z[m] = y1[bM + m] conj(y2[bM + m + L]), m < M. Its 128
// output columns are the real and imaginary parts of
// W_b(nu_q) = sum_m z[m] e^{j 2 pi nu_q m} on the snapshot's 64 bins. In real
// arithmetic, per 32-sample stage:
//     [z_re | z_im] (row, 64) x [[V_re, V_im], [-V_im, V_re]] (64, 128)
// The right-hand operand depends only on the snapshot, so it is precomputed
// once per snapshot in 16-bit (bf16 or fp16) in the tensor cores' canonical
// K-major layout and streamed into shared memory with bulk (TMA) copies. The
// lag products are formed on the CUDA cores and written into shared memory in
// the same layout.
//
// One CTA = 128 rows x 128 columns, the accumulator in tensor memory (128
// columns). Pipeline: two A buffers (while the tensor cores run stage j the
// CUDA cores fill stage j + 1) and three B buffers (the bulk copy of stage
// j + 1 is issued during stage j). A single thread issues the MMAs and commits
// them to an mbarrier. Each lane of the producer forms 8 consecutive lag
// products of one row and writes them as one 16-byte core-matrix row, so the
// shared-memory stores are conflict-free. The epilogue reads the accumulator with tcgen05.ld and writes
// W rows (planar: 64 real parts, then 64 imaginary parts) scaled back by
// 1 / zscale. Every mbarrier wait is bounded: on a timeout the kernel latches
// ERR_TIMEOUT, stops issuing, waits (bounded) for what it issued, frees its
// tensor memory and returns.
//
// Shared-memory operand layout (no swizzle, K-major): a 128-row x 32-element
// block is made of 8-row x 16-byte core matrices; element (row, k) is at byte
// ((row / 8) * 4 + k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2. K-adjacent
// core matrices are 128 B apart (the descriptor's leading byte offset) and
// 8-row groups 512 B apart (its stride byte offset).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "dg_internal.cuh"

namespace dg {
namespace {

constexpr int kRows = 128;                         // GEMM rows per CTA
constexpr int kN = 128;                            // 64 bins x (re, im)
constexpr int kKS = 32;                            // samples per stage
constexpr int kBlockBytes = kRows * kKS * 2;       // one 128 x 32 16-bit block
constexpr int kStages = 2;                         // A buffers (re, im blocks per part)
constexpr int kBStages = 3;                        // B buffers (re, im blocks per part), prefetched one stage ahead
// shared memory of a CTA for P 16-bit parts (1, or 2 for the split forms)
constexpr int smem_bytes(int P) { return (kStages + kBStages) * 2 * P * kBlockBytes; }
constexpr int kMmaThreads = 512;
constexpr uint32_t kWaitLimit = 1u << 24;          // try_wait polls before giving up

__device__ __forceinline__ uint32_t blk_off(int row, int k)
{
    return (uint32_t)(((row >> 3) * 4 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start >> 4 [0,14), LBO >> 4 [16,30),
// SBO >> 4 [32,46), version 1 [46,48), no swizzle [61,64).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) |
           (1ull << 46);
}

// Instruction descriptor, kind::f16: D f32 [4,6) = 1; A, B type [7,10), [10,13)
// (bf16 = 1, f16 = 0); both K-major; N >> 3 at [17,23); M >> 4 at [24,29).
template <int DT> __device__ __forceinline__ uint32_t idesc()
{
    const uint32_t t = DT == DG_CONTRACT_BF16 ? 1u : 0u;
    return (1u << 4) | (t << 7) | (t << 10) | ((uint32_t)(kN >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(ad), "l"(bd), "r"(id), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 consecutive 32-bit columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int DT> __device__ __forceinline__ uint32_t pack2(float a, float b);
template <> __device__ __forceinline__ uint32_t pack2<DG_CONTRACT_BF16>(float a, float b)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);  // a at the lower address
    return *reinterpret_cast<const uint32_t *>(&v);
}
template <> __device__ __forceinline__ uint32_t pack2<DG_CONTRACT_FP16>(float a, float b)
{
    const __half2 v = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&v);
}

template <int DT> __device__ __forceinline__ uint16_t to16(float a);
template <> __device__ __forceinline__ uint16_t to16<DG_CONTRACT_BF16>(float a)
{
    const __nv_bfloat16 v = __float2bfloat16_rn(a);
    return *reinterpret_cast<const uint16_t *>(&v);
}
template <> __device__ __forceinline__ uint16_t to16<DG_CONTRACT_FP16>(float a)
{
    const __half v = __float2half_rn(a);
    return *reinterpret_cast<const uint16_t *>(&v);
}

template <int DT> __device__ __forceinline__ float from16(uint16_t h);
template <> __device__ __forceinline__ float from16<DG_CONTRACT_BF16>(uint16_t h)
{
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(&h));
}
template <> __device__ __forceinline__ float from16<DG_CONTRACT_FP16>(uint16_t h)
{
    return __half2float(*reinterpret_cast<const __half *>(&h));
}

// Step of the batch owning tile t (tbase[s] <= t < tbase[s+1]).
__device__ __forceinline__ int step_of_tile(const int *base, int S, int t)
{
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace

// B operand of every snapshot: btab[s][j][part][blk][blk_off(n, k)] for
// 32-sample stage j, part 0 (high) / 1 (residual, split forms only), blk 0
// (multiplies z_re) / 1 (multiplies z_im), output column n, sample m = 32 j + k,
// bin q = n % 64, V = e^{j 2 pi (nubase + q delta) m}.
template <int DT, int P>
__global__ void __launch_bounds__(256) k_cdft_btab(const float *nubase, const float *delta, int M, uint16_t *btab)
{
    const int s = blockIdx.y;
    const int NJ = M / kKS;
    const size_t per_stage = (size_t)P * 2 * kRows * kKS;  // 16-bit elements
    const size_t per_step = (size_t)NJ * per_stage;
    const double b0 = (double)nubase[s], d = (double)delta[s];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)NJ * 2 * kRows * kKS;
         i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % kKS);
        const int n = (int)((i / kKS) % kRows);
        const int blk = (int)((i / (kKS * kRows)) % 2);
        const int j = (int)(i / (2 * kKS * kRows));
        const int m = j * kKS + k, q = n & 63;
        const double ph = (b0 + d * (double)q) * (double)m;
        float sn, cs;
        sincospif(2.0f * (float)(ph - floor(ph)), &sn, &cs);
        float v;
        if (blk == 0) v = n < 64 ? cs : sn;   // z_re * (V_re | V_im)
        else v = n < 64 ? -sn : cs;           // z_im * (-V_im | V_re)
        uint16_t *dst = btab + (size_t)s * per_step + (size_t)j * per_stage + blk_off(n, k) / 2;
        const uint16_t h = to16<DT>(v);
        dst[(size_t)blk * (kBlockBytes / 2)] = h;
        if (P == 2) dst[(size_t)(2 + blk) * (kBlockBytes / 2)] = to16<DT>(v - from16<DT>(h));
    }
}

// 8 consecutive samples starting at a multiple of 8, as floats.
template <int FMT> __device__ __forceinline__ void load8_aligned(const void *base, int idx, float2 (&v)[8]);
template <> __device__ __forceinline__ void load8_aligned<DG_IQ_C64>(const void *base, int idx, float2 (&v)[8])
{
    const float4 *p = reinterpret_cast<const float4 *>(base) + idx / 2;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 q = __ldg(p + i);
        v[2 * i] = make_float2(q.x, q.y);
        v[2 * i + 1] = make_float2(q.z, q.w);
    }
}
template <> __device__ __forceinline__ void load8_aligned<DG_IQ_CI16>(const void *base, int idx, float2 (&v)[8])
{
    const int4 *p = reinterpret_cast<const int4 *>(base) + idx / 4;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int4 q = __ldg(p + i);
        const int w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) v[4 * i + u] = make_float2((float)(short)(w[u] & 0xffff), (float)(short)(w[u] >> 16));
    }
}
template <> __device__ __forceinline__ void load8_aligned<DG_IQ_CI8>(const void *base, int idx, float2 (&v)[8])
{
    const int4 q = __ldg(reinterpret_cast<const int4 *>(base) + idx / 8);
    const int w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        v[2 * u] = make_float2((float)(signed char)(w[u] & 0xff), (float)(signed char)((w[u] >> 8) & 0xff));
        v[2 * u + 1] = make_float2((float)(signed char)((w[u] >> 16) & 0xff), (float)(signed char)(w[u] >> 24));
    }
}

// 8 consecutive samples starting at any index i0 with [i0, i0 + 8) inside
// [0, N): aligned 16-byte loads of the covering window, then a register
// shift. Falls back to bounded scalar loads when the aligned window would
// leave [0, N).
template <int FMT> __device__ __forceinline__ void load8_any(const void *base, int i0, int N, float2 (&v)[8]);

template <> __device__ __forceinline__ void load8_any<DG_IQ_CI16>(const void *base, int i0, int N, float2 (&v)[8])
{
    const int a0 = i0 & ~3, sh = i0 - a0;  // 4 samples per 16 bytes
    if (a0 >= 0 && a0 + 12 <= N) {
        const int4 *p = reinterpret_cast<const int4 *>(base) + (a0 >> 2);
        const int4 q0 = __ldg(p), q1 = __ldg(p + 1), q2 = __ldg(p + 2);
        const int w[12] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
        int o[8];
        switch (sh) {
        case 0:
#pragma unroll
            for (int u = 0; u < 8; ++u) o[u] = w[u];
            break;
        case 1:
#pragma unroll
            for (int u = 0; u < 8; ++u) o[u] = w[u + 1];
            break;
        case 2:
#pragma unroll
            for (int u = 0; u < 8; ++u) o[u] = w[u + 2];
            break;
        default:
#pragma unroll
            for (int u = 0; u < 8; ++u) o[u] = w[u + 3];
            break;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = make_float2((float)(short)(o[u] & 0xffff), (float)(short)(o[u] >> 16));
        return;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
        v[u] = (i0 + u >= 0 && i0 + u < N) ? IQ<DG_IQ_CI16>::load(base, i0 + u) : make_float2(0.f, 0.f);
}

template <> __device__ __forceinline__ void load8_any<DG_IQ_CI8>(const void *base, int i0, int N, float2 (&v)[8])
{
    const int a0 = i0 & ~7, sh = i0 - a0;  // 8 samples per 16 bytes, 2 samples per word
    if (a0 >= 0 && a0 + 16 <= N) {
        const int4 *p = reinterpret_cast<const int4 *>(base) + (a0 >> 3);
        const int4 q0 = __ldg(p), q1 = __ldg(p + 1);
        const unsigned w[8] = {(unsigned)q0.x, (unsigned)q0.y, (unsigned)q0.z, (unsigned)q0.w,
                               (unsigned)q1.x, (unsigned)q1.y, (unsigned)q1.z, (unsigned)q1.w};
        // sample t of the window lives in half-word t of w; take half-words sh .. sh + 7
        const int wo = sh >> 1;
        unsigned o[4];
        if (sh & 1) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                unsigned lo_w = 0, hi_w = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (wo == c) {
                        lo_w = w[c + u];
                        hi_w = w[c + u + 1];
                    }
                o[u] = __byte_perm(lo_w, hi_w, 0x5432);
            }
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                unsigned x = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (wo == c) x = w[c + u];
                o[u] = x;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int x = (int)o[u];
            v[2 * u] = make_float2((float)(signed char)(x & 0xff), (float)(signed char)((x >> 8) & 0xff));
            v[2 * u + 1] = make_float2((float)(signed char)((x >> 16) & 0xff), (float)(signed char)(x >> 24));
        }
        return;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
        v[u] = (i0 + u >= 0 && i0 + u < N) ? IQ<DG_IQ_CI8>::load(base, i0 + u) : make_float2(0.f, 0.f);
}

template <> __device__ __forceinline__ void load8_any<DG_IQ_C64>(const void *base, int i0, int N, float2 (&v)[8])
{
    const int a0 = i0 & ~1, sh = i0 - a0;  // 2 samples per 16 bytes
    if (a0 >= 0 && a0 + 10 <= N) {
        const float4 *p = reinterpret_cast<const float4 *>(base) + (a0 >> 1);
        float2 w[10];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float4 q = __ldg(p + i);
            w[2 * i] = make_float2(q.x, q.y);
            w[2 * i + 1] = make_float2(q.z, q.w);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = sh ? w[u + 1] : w[u];
        return;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
        v[u] = (i0 + u >= 0 && i0 + u < N) ? IQ<DG_IQ_C64>::load(base, i0 + u) : make_float2(0.f, 0.f);
}

template <int FMT, int DT, int P>
__global__ void __launch_bounds__(kMmaThreads) k_cdft_contract_mma(CdftBatch a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_full[kBStages], bar_mma[kStages];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_last_commit;

    const int tile = blockIdx.x;
    const int s = step_of_tile(a.tbase, a.S, tile);
    const int ltile = tile - a.tbase[s];
    const StepDesc sd = a.sd[s];
    const int N = sd.n, M = a.M;
    const int Bs = (N + M - 1) / M;
    const int NB = a.bbase[s + 1] - a.bbase[s];
    const int64_t R = (int64_t)NB * Bs;
    const int NJ = M / kKS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // producer tasks: lane = 8 rows x 4 groups of 8 samples (lanes 0-7 take
    // group 0 of the warp's 8 rows, so each quarter-warp stores one 128-byte
    // line of core-matrix rows); warp w covers rows 8 w .. 8 w + 7
    const int rin = lane & 7, kg = lane >> 3;
    int pL[1], pn0[1];
    bool pv[1];
#pragma unroll
    for (int h = 0; h < 1; ++h) {
        const int row = 8 * warp + rin;
        const int64_t g = (int64_t)ltile * kRows + row;
        pv[h] = g < R;
        pL[h] = 0;
        pn0[h] = 0;
        if (pv[h]) {
            const int bl = (int)(g / Bs);
            pn0[h] = (int)(g % Bs) * M + 8 * kg;  // first sample of this lane at stage 0
            pL[h] = a.lr[2 * s] + bl;
            pv[h] = a.count[a.bbase[s] + bl] > 0;
        }
    }

    constexpr int kSt = 2 * P * kBlockBytes;  // bytes of one stage's A (or B) blocks
    unsigned char *sAbase = smem;
    unsigned char *sBbase = smem + kStages * kSt;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kBStages; ++i) mbar_init(smem_u32(&bar_full[i]), 1);
        for (int i = 0; i < kStages; ++i) mbar_init(smem_u32(&bar_mma[i]), 1);
        s_last_commit = -1;
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_slot), 128);
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_slot;
    const unsigned char *bsrc = reinterpret_cast<const unsigned char *>(a.btab) + (size_t)s * NJ * kSt;
    const float zs = a.zscale;
    bool aborted = false;  // meaningful in thread 0 (the issuer)
    if (threadIdx.x == 0) {  // B of stage 0
        mbar_expect_tx(smem_u32(&bar_full[0]), kSt);
        bulk_g2s(smem_u32(sBbase), bsrc, kSt, smem_u32(&bar_full[0]));
    }

    for (int j = 0; j < NJ; ++j) {
        const int st = j & 1, bt = j % kBStages;
        unsigned char *sA = sAbase + st * kSt;
        unsigned char *sB = sBbase + bt * kSt;
        bool bad = false;
        // the MMAs of stage j - 2 read A buffer st and B buffer (j + 1) % 3
        if (j >= 2) bad = !mbar_wait(smem_u32(&bar_mma[st]), (uint32_t)((j - 2) >> 1) & 1u);
        if (__syncthreads_or(bad || aborted)) {
            if (threadIdx.x == 0) atomicOr(a.err, ERR_TIMEOUT);
            aborted = true;
            break;
        }
        if (threadIdx.x == 0 && j + 1 < NJ) {  // prefetch B of stage j + 1
            const int nb = (j + 1) % kBStages;
            mbar_expect_tx(smem_u32(&bar_full[nb]), kSt);
            bulk_g2s(smem_u32(sBbase + nb * kSt), bsrc + (size_t)(j + 1) * kSt, kSt, smem_u32(&bar_full[nb]));
        }
        // lag products of 8 consecutive samples of one row, rounded to 16 bits
#pragma unroll
        for (int h = 0; h < 1; ++h) {
            const int row = 8 * warp + rin;
            float2 x[8];
            float zr[8], zi[8];
            const int n = pn0[h] + j * kKS;
            if (pv[h] && n + 8 <= N) {
                load8_aligned<FMT>(sd.y1, n, x);
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    x[u] = (pv[h] && n + u < N) ? IQ<FMT>::load(sd.y1, n + u) : make_float2(0.f, 0.f);
            }
            float2 y[8];
            if (pv[h]) {
                load8_any<FMT>(sd.y2, n + pL[h], N, y);
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) y[u] = make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                // samples beyond the end of y1 contribute nothing (x is zero there)
                zr[u] = fmaf(x[u].x, y[u].x, x[u].y * y[u].y) * zs;
                zi[u] = fmaf(x[u].y, y[u].x, -x[u].x * y[u].y) * zs;
            }
            uint16_t hr[8], hi[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                hr[u] = to16<DT>(zr[u]);
                hi[u] = to16<DT>(zi[u]);
            }
            auto pk = [](const uint16_t *h) {
                return make_uint4((uint32_t)h[0] | ((uint32_t)h[1] << 16), (uint32_t)h[2] | ((uint32_t)h[3] << 16),
                                  (uint32_t)h[4] | ((uint32_t)h[5] << 16), (uint32_t)h[6] | ((uint32_t)h[7] << 16));
            };
            *reinterpret_cast<uint4 *>(sA + blk_off(row, 8 * kg)) = pk(hr);
            *reinterpret_cast<uint4 *>(sA + kBlockBytes + blk_off(row, 8 * kg)) = pk(hi);
            if (P == 2) {  // residuals z - high part, rounded to 16 bits
                uint16_t lr[8], li[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    lr[u] = to16<DT>(zr[u] - from16<DT>(hr[u]));
                    li[u] = to16<DT>(zi[u] - from16<DT>(hi[u]));
                }
                *reinterpret_cast<uint4 *>(sA + 2 * kBlockBytes + blk_off(row, 8 * kg)) = pk(lr);
                *reinterpret_cast<uint4 *>(sA + 3 * kBlockBytes + blk_off(row, 8 * kg)) = pk(li);
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            if (!mbar_wait(smem_u32(&bar_full[bt]), (uint32_t)(j / kBStages) & 1u)) {
                aborted = true;  // reported at the top of the next iteration / after the loop
            } else {
                tc_after_sync();
                const uint32_t id = idesc<DT>();
                // products per block: high x high, and for the split forms also
                // residual x high and high x residual (part p at p * 2 blocks)
                constexpr int NPROD = P == 2 ? 3 : 1;
#pragma unroll
                for (int blk = 0; blk < 2; ++blk)
#pragma unroll
                    for (int kk = 0; kk < kKS; kk += 16)
#pragma unroll
                        for (int pr = 0; pr < NPROD; ++pr) {
                            const int pa = pr == 1 ? 1 : 0, pb = pr == 2 ? 1 : 0;
                            const uint64_t ad = sdesc(smem_u32(sA + (2 * pa + blk) * kBlockBytes) + kk * 16);
                            const uint64_t bd = sdesc(smem_u32(sB + (2 * pb + blk) * kBlockBytes) + kk * 16);
                            mma_f16(tmem, ad, bd, id, (j > 0 || blk > 0 || kk > 0 || pr > 0) ? 1u : 0u);
                        }
                mma_commit(smem_u32(&bar_mma[st]));
                s_last_commit = j;
            }
        }
    }
    // the last commit covers every MMA this CTA issued
    __syncthreads();
    const int lc = s_last_commit;
    bool ok = lc >= 0 && mbar_wait(smem_u32(&bar_mma[lc & 1]), (uint32_t)(lc >> 1) & 1u);
    if (threadIdx.x == 0 && aborted) atomicOr(a.err, ERR_TIMEOUT);
    ok = !__syncthreads_or(!ok || aborted || lc != NJ - 1);
    tc_after_sync();
    if (ok) {
        // warp w reads lanes 32 (w % 4) .. +31 (its rows), columns 32 (w / 4) .. +31
        const int row = 32 * (warp & 3) + lane, quarter = warp >> 2;
        const int64_t g = (int64_t)ltile * kRows + row;
        bool valid = g < R;
        int64_t wrow = 0;
        if (valid) {
            const int bl = (int)(g / Bs);
            valid = a.count[a.bbase[s] + bl] > 0;
            wrow = ((int64_t)(a.bbase[s] + bl) * a.Bmax + g % Bs) * 128;
        }
        const float inv = 1.0f / zs;
        const uint32_t tbase = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * quarter);
        {
            const int c = 0;
            uint32_t r[32];
            tmem_ld32(tbase, r);
            if (valid) {
                float4 *w = reinterpret_cast<float4 *>(a.W + wrow + 32 * quarter + c);
#pragma unroll
                for (int v = 0; v < 8; ++v)
                    w[v] = make_float4(__uint_as_float(r[4 * v]) * inv, __uint_as_float(r[4 * v + 1]) * inv,
                                       __uint_as_float(r[4 * v + 2]) * inv, __uint_as_float(r[4 * v + 3]) * inv);
            }
        }
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 128);
}

cudaError_t launch_cdft_btab(const CdftBatch &a, int mode, void *btab, cudaStream_t st)
{
    const size_t n = (size_t)(a.M / kKS) * 2 * kRows * kKS;
    unsigned gx = (unsigned)std::min<size_t>((n + 255) / 256, 1024);
    dim3 grid(gx, (unsigned)a.S);
    switch (mode) {
    case DG_CONTRACT_BF16: k_cdft_btab<DG_CONTRACT_BF16, 1><<<grid, 256, 0, st>>>(a.nubase, a.delta, a.M, (uint16_t *)btab); break;
    case DG_CONTRACT_FP16: k_cdft_btab<DG_CONTRACT_FP16, 1><<<grid, 256, 0, st>>>(a.nubase, a.delta, a.M, (uint16_t *)btab); break;
    case DG_CONTRACT_BF16X3: k_cdft_btab<DG_CONTRACT_BF16, 2><<<grid, 256, 0, st>>>(a.nubase, a.delta, a.M, (uint16_t *)btab); break;
    default: k_cdft_btab<DG_CONTRACT_FP16, 2><<<grid, 256, 0, st>>>(a.nubase, a.delta, a.M, (uint16_t *)btab); break;
    }
    return cudaGetLastError();
}

size_t cdft_btab_bytes(int mode, int M) { return (size_t)(M / kKS) * 2 * (mode >= DG_CONTRACT_BF16X3 ? 2 : 1) * kBlockBytes; }

template <int FMT, int DT, int P>
static cudaError_t launch_mma(const CdftBatch &a, int tiles, cudaStream_t st)
{
    const int smem = smem_bytes(P);
    cudaError_t e = cudaFuncSetAttribute(k_cdft_contract_mma<FMT, DT, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_cdft_contract_mma<FMT, DT, P><<<(unsigned)tiles, kMmaThreads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int DT, int P>
static cudaError_t launch_fmt(const CdftBatch &a, int tiles, int fmt, cudaStream_t st)
{
    switch (fmt) {
    case DG_IQ_C64: return launch_mma<DG_IQ_C64, DT, P>(a, tiles, st);
    case DG_IQ_CI16: return launch_mma<DG_IQ_CI16, DT, P>(a, tiles, st);
    default: return launch_mma<DG_IQ_CI8, DT, P>(a, tiles, st);
    }
}

cudaError_t launch_cdft_contract_mma(const CdftBatch &a, int tiles, int fmt, int mode, cudaStream_t st)
{
    switch (mode) {
    case DG_CONTRACT_BF16: return launch_fmt<DG_CONTRACT_BF16, 1>(a, tiles, fmt, st);
    case DG_CONTRACT_FP16: return launch_fmt<DG_CONTRACT_FP16, 1>(a, tiles, fmt, st);
    case DG_CONTRACT_BF16X3: return launch_fmt<DG_CONTRACT_BF16, 2>(a, tiles, fmt, st);
    default: return launch_fmt<DG_CONTRACT_FP16, 2>(a, tiles, fmt, st);
    }
}

}  // namespace dg
