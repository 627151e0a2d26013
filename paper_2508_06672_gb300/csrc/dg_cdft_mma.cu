// dg_cdft_mma.cu -- the chunked-DFT contraction on the 5th-generation tensor
// cores (tcgen05, sm_103a), 16-bit products accumulated in FP32.
//
// For one snapshot the contraction is one tall GEMM. Its rows are the
// (lag bucket, chunk) pairs. For chunk b of lag L the row holds the lag
// products z[m] = y1[bM + m] conj(y2[bM + m + L]), m < M; its 128 output
// columns are the real and imaginary parts of W_b(nu_q) = sum_m z[m]
// e^{j 2 pi nu_q m} on the snapshot's 64 bins. In real arithmetic, per
// 32-sample stage:
//     [z_re | z_im] (row, 64) x [[V_re, V_im], [-V_im, V_re]] (64, 128)
// The right-hand operand depends only on the snapshot: k_cdft_btab writes it
// once per snapshot in 16 bits (bf16 or fp16; high part and residual for the
// split forms) in the tensor cores' canonical K-major layout, and the
// contraction streams it into shared memory with bulk (TMA) copies.
//
// k_cdft_contract_tc is persistent: one CTA of 704 threads per SM walks the
// batch's tiles (blockIdx.x, + gridDim.x, ...), each 128 rows x 128 columns,
// laid out on the device by k_cdft_tiles. A tile is either 128 consecutive
// lags at one chunk (lag tiles: the chunk's y1 and the y2 window of the 128
// lags are staged in shared memory, in windows of 1024 samples, the next
// window prefetched into registers while the current one's stages run) or
// 128 consecutive (lag, chunk) rows (row tiles: each lane loads its row's
// capture segments). Roles:
//   16 producer warps  form the lag products of each stage (lane l of warp w
//                      takes row 32 (w % 4) + l, 8 samples; a warp reaches
//                      only its quarter of the tensor-memory lanes) and store
//                      them with tcgen05.st into a ring of 4 A stages in
//                      tensor memory; a stage's arrival on its "A full"
//                      barrier follows the next stage's math, so the stores
//                      land meanwhile;
//   1 loader thread    streams the DFT operand into a ring of 5 shared-memory
//                      stages (complete_tx barriers), across tiles;
//   1 MMA thread       issues tcgen05.mma kind::f16 (A from tensor memory, B
//                      from shared memory; three products per K step for the
//                      split forms) and commits them to the stages' "empty"
//                      barriers and, at a tile's end, to its accumulator;
//   4 epilogue warps   drain each finished accumulator (tcgen05.ld) into W
//                      rows (planar: 64 real parts, then 64 imaginary parts,
//                      scaled back by 1 / zscale) while the next tile's MMAs
//                      run in the other of the two 128-column accumulators.
// Every mbarrier wait is bounded (2 s of the global timer, or a poll limit).
// On a timeout the CTA latches ERR_TIMEOUT and every role stops issuing; the
// loader waits for its copies in flight and the MMA thread commits to a last
// barrier that completes when its MMAs have, which is waited for before the
// tensor memory is freed and the CTA returns.
//
// Shared-memory operand layout (no swizzle, K-major): a 128-row x 32-element
// block is made of 8-row x 16-byte core matrices; element (row, k) is at byte
// ((row / 8) * 4 + k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2. K-adjacent
// core matrices are 128 B apart (the descriptor's leading byte offset) and
// 8-row groups 512 B apart (its stride byte offset).
//
// k_cdft_contract_hk (Hankel tiles, on request) regroups the product so that
// y2 itself is the right operand; see its own comment below.
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
constexpr uint32_t kWaitLimit = 1u << 24;          // try_wait polls before giving up
constexpr uint64_t kWaitBudgetNs = 2000000000ull;  // and the clock budget of one wait (2 s)

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

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase: gives up after kWaitBudgetNs of the
// global timer (checked every 256 polls) or kWaitLimit polls, whichever
// comes first (try_wait may suspend the thread for a while per poll). The
// pipeline's waits take a lower poll limit when one is set for tests
// (CdftBatch::wait_polls); the waits that drain an aborted pipeline always
// take the full limit.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit = kWaitLimit)
{
    uint64_t t0 = 0;
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((i & 255) == 255) {
            const uint64_t now = globaltimer_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > kWaitBudgetNs) return false;
        }
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

// The same MMA with A in tensor memory (128 lanes = rows, K along columns,
// two 16-bit elements per 32-bit column, the even one in the low half).
__device__ __forceinline__ void mma_f16_ta(uint32_t d, uint32_t at, uint64_t bd, uint32_t id, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
        "r"(at), "l"(bd), "r"(id), "r"(acc)
        : "memory");
}

// 4 consecutive 32-bit columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t (&r)[4])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(r[0]), "r"(r[1]),
                 "r"(r[2]), "r"(r[3])
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

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

template <int DT> __device__ __forceinline__ float2 unpack2(uint32_t v);
template <> __device__ __forceinline__ float2 unpack2<DG_CONTRACT_BF16>(uint32_t v)
{
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v));
}
template <> __device__ __forceinline__ float2 unpack2<DG_CONTRACT_FP16>(uint32_t v)
{
    return __half22float2(*reinterpret_cast<const __half2 *>(&v));
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
//
// One thread per (bin q, stage j, 8 consecutive samples): one sin/cos per
// (q, m) serves the four entries it feeds -- (blk 0, n = q) V_re,
// (blk 0, n = q + 64) V_im, (blk 1, n = q) -V_im, (blk 1, n = q + 64) V_re --
// and each lands as one 16-byte row of a core matrix.
template <int DT, int P>
__device__ __forceinline__ void btab_row(uint16_t *stage, int blk, int n, int kg, const float (&v)[8], float sign)
{
    uint32_t h[4], r[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float x0 = sign * v[2 * e], x1 = sign * v[2 * e + 1];
        const uint16_t h0 = to16<DT>(x0), h1 = to16<DT>(x1);
        h[e] = (uint32_t)h0 | ((uint32_t)h1 << 16);
        if (P == 2)
            r[e] = (uint32_t)to16<DT>(x0 - from16<DT>(h0)) | ((uint32_t)to16<DT>(x1 - from16<DT>(h1)) << 16);
    }
    uint16_t *dst = stage + blk_off(n, 8 * kg) / 2;
    *reinterpret_cast<uint4 *>(dst + (size_t)blk * (kBlockBytes / 2)) = make_uint4(h[0], h[1], h[2], h[3]);
    if (P == 2)
        *reinterpret_cast<uint4 *>(dst + (size_t)(2 + blk) * (kBlockBytes / 2)) = make_uint4(r[0], r[1], r[2], r[3]);
}

template <int DT, int P>
__global__ void __launch_bounds__(256) k_cdft_btab(const float *nubase, const float *delta, int M, uint16_t *btab)
{
    const int s = blockIdx.y;
    const int NJ = M / kKS;
    const size_t per_stage = (size_t)P * 2 * kRows * kKS;  // 16-bit elements
    const size_t per_step = (size_t)NJ * per_stage;
    const float b0 = nubase[s], d = delta[s];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)NJ * 64 * (kKS / 8);
         i += (size_t)gridDim.x * blockDim.x) {
        const int kg = (int)(i % (kKS / 8));
        const int q = (int)((i / (kKS / 8)) % 64);
        const int j = (int)(i / (64 * (kKS / 8)));
        // bin frequency in FP32 as the combine forms it; the phase of
        // sample m (< 2^24) from the exact product split
        const float fq = fmaf((float)q, d, b0);
        float sn[8], cs[8];
#pragma unroll
        for (int e = 0; e < 8; ++e)
            sincospif(2.0f * frac_mul(fq, (float)(j * kKS + 8 * kg + e)), &sn[e], &cs[e]);
        uint16_t *stage = btab + (size_t)s * per_step + (size_t)j * per_stage;
        btab_row<DT, P>(stage, 0, q, kg, cs, 1.0f);        // z_re * V_re
        btab_row<DT, P>(stage, 0, q + 64, kg, sn, 1.0f);   // z_re * V_im
        btab_row<DT, P>(stage, 1, q, kg, sn, -1.0f);       // z_im * (-V_im)
        btab_row<DT, P>(stage, 1, q + 64, kg, cs, 1.0f);   // z_im * V_re
    }
}

// Raw loads of one lane's 8 samples of y1 (index n, a multiple of 8) and of
// y2 (index n2, any) for a stage, issued one stage ahead and decoded when
// used. The aligned 16-byte windows are only loaded when they lie inside
// [0, N); otherwise decode() reads the samples one by one with bounds.
template <int FMT> struct Raw;

template <> struct Raw<DG_IQ_CI16> {
    int4 a[2], b[3];
    int n, n2;
    bool f1, f2;
    __device__ __forceinline__ void fetch(const void *y1, const void *y2, int n_, int n2_, int N, bool v)
    {
        n = n_;
        n2 = n2_;
        const int a0 = n2 & ~3;
        f1 = v && n + 8 <= N;
        f2 = v && a0 >= 0 && a0 + 12 <= N;
        if (f1) {
            const int4 *p = reinterpret_cast<const int4 *>(y1) + (n >> 2);
            a[0] = __ldg(p);
            a[1] = __ldg(p + 1);
        }
        if (f2) {
            const int4 *p = reinterpret_cast<const int4 *>(y2) + (a0 >> 2);
            b[0] = __ldg(p);
            b[1] = __ldg(p + 1);
            b[2] = __ldg(p + 2);
        }
    }
    __device__ __forceinline__ void decode(const void *y1, const void *y2, int N, bool v, float2 (&x)[8],
                                           float2 (&y)[8]) const
    {
        if (f1) {
            const int w[8] = {a[0].x, a[0].y, a[0].z, a[0].w, a[1].x, a[1].y, a[1].z, a[1].w};
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = make_float2((float)(short)(w[u] & 0xffff), (float)(short)(w[u] >> 16));
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u)
                x[u] = (v && n + u < N) ? IQ<DG_IQ_CI16>::load(y1, n + u) : make_float2(0.f, 0.f);
        }
        if (f2) {
            const int w[12] = {b[0].x, b[0].y, b[0].z, b[0].w, b[1].x, b[1].y, b[1].z, b[1].w,
                               b[2].x, b[2].y, b[2].z, b[2].w};
            const int sh = n2 & 3;
            int o[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) o[u] = sh == 0 ? w[u] : sh == 1 ? w[u + 1] : sh == 2 ? w[u + 2] : w[u + 3];
#pragma unroll
            for (int u = 0; u < 8; ++u) y[u] = make_float2((float)(short)(o[u] & 0xffff), (float)(short)(o[u] >> 16));
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u)
                y[u] = (v && n2 + u >= 0 && n2 + u < N) ? IQ<DG_IQ_CI16>::load(y2, n2 + u) : make_float2(0.f, 0.f);
        }
    }
};

template <> struct Raw<DG_IQ_CI8> {
    int4 a, b[2];
    int n, n2;
    bool f1, f2;
    __device__ __forceinline__ void fetch(const void *y1, const void *y2, int n_, int n2_, int N, bool v)
    {
        n = n_;
        n2 = n2_;
        const int a0 = n2 & ~7;
        f1 = v && n + 8 <= N;
        f2 = v && a0 >= 0 && a0 + 16 <= N;
        if (f1) a = __ldg(reinterpret_cast<const int4 *>(y1) + (n >> 3));
        if (f2) {
            const int4 *p = reinterpret_cast<const int4 *>(y2) + (a0 >> 3);
            b[0] = __ldg(p);
            b[1] = __ldg(p + 1);
        }
    }
    static __device__ __forceinline__ void unpack(const unsigned (&o)[4], float2 (&v)[8])
    {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int x = (int)o[u];
            v[2 * u] = make_float2((float)(signed char)(x & 0xff), (float)(signed char)((x >> 8) & 0xff));
            v[2 * u + 1] = make_float2((float)(signed char)((x >> 16) & 0xff), (float)(signed char)(x >> 24));
        }
    }
    __device__ __forceinline__ void decode(const void *y1, const void *y2, int N, bool v, float2 (&x)[8],
                                           float2 (&y)[8]) const
    {
        if (f1) {
            const unsigned o[4] = {(unsigned)a.x, (unsigned)a.y, (unsigned)a.z, (unsigned)a.w};
            unpack(o, x);
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u)
                x[u] = (v && n + u < N) ? IQ<DG_IQ_CI8>::load(y1, n + u) : make_float2(0.f, 0.f);
        }
        if (f2) {
            const unsigned w[8] = {(unsigned)b[0].x, (unsigned)b[0].y, (unsigned)b[0].z, (unsigned)b[0].w,
                                   (unsigned)b[1].x, (unsigned)b[1].y, (unsigned)b[1].z, (unsigned)b[1].w};
            // sample t of the window is half-word t of w; take half-words sh .. sh + 7
            const int sh = n2 & 7, wo = sh >> 1;
            unsigned o[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                unsigned lo_w = 0, hi_w = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (wo == c) {
                        lo_w = w[c + u];
                        hi_w = w[c + u + 1];
                    }
                o[u] = (sh & 1) ? __byte_perm(lo_w, hi_w, 0x5432) : lo_w;
            }
            unpack(o, y);
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u)
                y[u] = (v && n2 + u >= 0 && n2 + u < N) ? IQ<DG_IQ_CI8>::load(y2, n2 + u) : make_float2(0.f, 0.f);
        }
    }
};

template <> struct Raw<DG_IQ_C64> {
    float4 a[4], b[5];
    int n, n2;
    bool f1, f2;
    __device__ __forceinline__ void fetch(const void *y1, const void *y2, int n_, int n2_, int N, bool v)
    {
        n = n_;
        n2 = n2_;
        const int a0 = n2 & ~1;
        f1 = v && n + 8 <= N;
        f2 = v && a0 >= 0 && a0 + 10 <= N;
        if (f1) {
            const float4 *p = reinterpret_cast<const float4 *>(y1) + (n >> 1);
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = __ldg(p + i);
        }
        if (f2) {
            const float4 *p = reinterpret_cast<const float4 *>(y2) + (a0 >> 1);
#pragma unroll
            for (int i = 0; i < 5; ++i) b[i] = __ldg(p + i);
        }
    }
    __device__ __forceinline__ void decode(const void *y1, const void *y2, int N, bool v, float2 (&x)[8],
                                           float2 (&y)[8]) const
    {
        if (f1) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                x[2 * i] = make_float2(a[i].x, a[i].y);
                x[2 * i + 1] = make_float2(a[i].z, a[i].w);
            }
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u)
                x[u] = (v && n + u < N) ? IQ<DG_IQ_C64>::load(y1, n + u) : make_float2(0.f, 0.f);
        }
        if (f2) {
            float2 w[10];
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                w[2 * i] = make_float2(b[i].x, b[i].y);
                w[2 * i + 1] = make_float2(b[i].z, b[i].w);
            }
            const bool sh = n2 & 1;
#pragma unroll
            for (int u = 0; u < 8; ++u) y[u] = sh ? w[u + 1] : w[u];
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u)
                y[u] = (v && n2 + u >= 0 && n2 + u < N) ? IQ<DG_IQ_C64>::load(y2, n2 + u) : make_float2(0.f, 0.f);
        }
    }
};

// Warp-specialised pipeline. Producer warps write A (lag products) into a
// ring of ring_a<P>() slots; one control thread streams B (the DFT operand)
// by bulk copy into a ring of ring_b<P>() slots and issues the MMAs. Per slot:
// full_a (one arrival per producer warp) / full_b (bulk-copy bytes), and
// empty_a / empty_b (tcgen05.commit of the MMAs that read the slot).
constexpr int kProducerWarps = 16;  // enough warps per scheduler to hide the producers' load-math-store latency
constexpr int kRowSets = kRows / (8 * kProducerWarps);  // 8-row sets per producer warp
constexpr int kEpilogueWarps = 4;  // one per 32-lane quarter of the accumulator
constexpr int kSnapCache = kTcMaxSnapshots;  // per-snapshot tables cached in shared memory
// warps: producers, then the MMA thread's warp, the operand loader's warp,
// then the epilogue warps
constexpr int kMmaWarp = kProducerWarps, kLoadWarp = kProducerWarps + 1;
constexpr int kWsThreads = (kProducerWarps + 2 + kEpilogueWarps) * 32;
template <int P> __host__ __device__ constexpr int ring_a() { return P == 2 ? 4 : 8; }
template <int P> __host__ __device__ constexpr int ring_b() { return P == 2 ? 5 : 10; }
template <int P> __host__ __device__ constexpr int ws_smem_bytes()
{
    return ring_b<P>() * (2 * P * kBlockBytes);  // the A stages live in tensor memory
}
// tensor memory: two accumulators of 128 columns, then the A ring, each stage
// (high, residual) x (re, im) blocks of 16 columns (32 samples)
constexpr int kAccCols = 256;
template <int P> __host__ __device__ constexpr int a_stage_cols() { return 2 * P * 16; }
static_assert(kAccCols + ring_a<2>() * a_stage_cols<2>() <= 512 && kAccCols + ring_a<1>() * a_stage_cols<1>() <= 512,
              "accumulators and the A ring must fit the 512 tensor-memory columns");

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Lag buckets of snapshot s in this batch (0 if it has no representable lag).
__device__ __forceinline__ int nb_of(const CdftBatch &a, int s)
{
    const int lo = a.lr[2 * s], hi = a.lr[2 * s + 1];
    return hi >= lo ? hi - lo + 1 : 0;
}

// Persistent, warp-specialised contraction over every tile of the batch.
// The tile list (tbase, per-snapshot layout) is computed on the device by
// k_cdft_tiles, so the host launches a fixed grid without knowing it; the
// per-snapshot tables (at most kSnapCache snapshots per batch) are cached in
// shared memory. Each CTA walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...;
// a tile is either
//   rows: 128 consecutive (lag, chunk) rows, lag-major; each producer lane
//         loads its row's capture segments (Raw<FMT>), or
//   lags: 128 consecutive lags L0 .. L0 + 127 at one chunk b; the producers
//         stage y1[bM .. bM + M) (scaled by zscale) and the window
//         y2[bM + L0 .. bM + L0 + M + 127) in shared memory, decoded to FP32,
//         and then read only shared memory.
// Samples outside [0, N) are zero in both, so the sums run over the overlap.
// Roles:
//   warps 0-15 produce the lag products of each stage into a ring of
//              ring_a<P>() slots;
//   warp 16    (one thread) issues the MMAs of each stage once its A and B
//              are in, and commits them to the stage's empty barriers;
//   warp 17    (one thread) streams the DFT operand by bulk copy, up to
//              ring_b<P>() stages ahead of the MMAs, across tiles;
//   warps 18-21 drain each finished accumulator (tcgen05.ld -> W) while the
//              next tile's MMAs run.
// Two accumulators of 128 TMEM columns alternate between tiles. Every
// mbarrier keeps one phase sequence for the CTA's lifetime; every wait is
// bounded (mbar_wait); a timeout stops all roles, latches ERR_TIMEOUT, and the
// CTA frees its TMEM after waiting (bounded) for the MMAs it issued.
template <int P> __host__ __device__ constexpr int tc_smem_bytes()
{
    return ws_smem_bytes<P>() + (2 * kLagTileMaxChunk + kRows) * (int)sizeof(float2);
}

struct SnapCache {  // per-snapshot tables of the batch, in shared memory
    int tbase[kSnapCache + 1];
    int bbase[kSnapCache + 1];
    int lr[2 * kSnapCache];
    int layout[kSnapCache];
    StepDesc sd[kSnapCache];
};

struct TileInfo {
    int s, ltile, N, Bs, NB, lay, lb, bch, Lmin, bb;
    int rt, rNB, rl0;  // row tiles: tile index among them, their lags, first lag bucket
    int M, job;        // the job's chunk, and the job (0 in a single-job launch)
    StepDesc sd;
};

// A job's per-snapshot tables, in shared memory (the single job of a launch,
// cached) or in global memory (a launch over several jobs).
struct JobTables {
    const int *tbase, *bbase, *lr, *layout;
    const StepDesc *sd;
};

__device__ __forceinline__ TileInfo tile_info(const JobTables &c, int S, int M, int tile)
{
    TileInfo t;
    t.M = M;
    t.job = 0;
    t.s = step_of_tile(c.tbase, S, tile);
    t.ltile = tile - c.tbase[t.s];
    t.sd = c.sd[t.s];
    t.N = t.sd.n;
    t.Bs = (t.N + M - 1) / M;
    const int lo = c.lr[2 * t.s], hi = c.lr[2 * t.s + 1];
    t.NB = hi >= lo ? hi - lo + 1 : 0;
    // layout 0: row tiles over every lag; 1: lag tiles over every lag;
    // 3 (mixed): lag tiles over the whole blocks of 128 lags, then row tiles
    // over the remaining lags; t.lay is this tile's kind (1 lags, 0 rows)
    const int lay = c.layout[t.s];
    t.lay = lay == 1 ? 1 : 0;
    t.lb = t.bch = 0;
    t.rt = t.ltile;
    t.rNB = t.NB;
    t.rl0 = 0;
    if (lay == 1) {
        const int NLB = max((t.NB + kRows - 1) / kRows, 1);
        t.lb = t.ltile % NLB;
        t.bch = t.ltile / NLB;
    } else if (lay == 3) {
        const int NFB = max(t.NB / kRows, 1), nlt = NFB * t.Bs;
        if (t.ltile < nlt) {
            t.lay = 1;
            t.lb = t.ltile % NFB;
            t.bch = t.ltile / NFB;
        } else {
            t.rt = t.ltile - nlt;
            t.rl0 = NFB * kRows;
            t.rNB = max(t.NB - t.rl0, 0);
        }
    }
    t.Lmin = lo;
    t.bb = c.bbase[t.s];
    return t;
}

// A lag tile's chunk is staged in windows of SW = min(M, kLagTileMaxChunk)
// samples (M is then a multiple of SW): window w holds y1[n0 .. n0 + SW) and
// y2[n0 + L0 .. n0 + L0 + SW + 127), n0 = bch M + w SW.
__device__ __forceinline__ int window_len(int M) { return M < kLagTileMaxChunk ? M : kLagTileMaxChunk; }

// Window w of a lag tile into shared memory, by `nthreads` threads from `tid`.
template <int FMT>
__device__ __forceinline__ void stage_windows(const TileInfo &t, int M, int w, float zs, float2 *sy1, float2 *sy2,
                                              int tid, int nthreads)
{
    const int SW = window_len(M);
    const int nb0 = t.bch * M + w * SW, L0 = t.Lmin + t.lb * kRows;
    for (int i = tid; i < SW; i += nthreads) {
        const int n = nb0 + i;
        const float2 v = n < t.N ? IQ<FMT>::load(t.sd.y1, n) : make_float2(0.f, 0.f);
        sy1[i] = make_float2(v.x * zs, v.y * zs);
    }
    for (int i = tid; i < SW + kRows; i += nthreads) {
        const int n2 = nb0 + L0 + i;
        sy2[i] = (n2 >= 0 && n2 < t.N) ? IQ<FMT>::load(t.sd.y2, n2) : make_float2(0.f, 0.f);
    }
}

// The next window (of this lag tile or of the next one), prefetched into the
// producers' registers while the current window's stages run: element e of
// thread tid is window element tid + 512 e (y1[n0 + i] for i < SW, then
// y2[n0 + L0 + i - SW]), kept raw (2, 4 or 8 bytes) and decoded only when
// the window starts.
constexpr int kPfPer = (2 * kLagTileMaxChunk + kRows + kProducerWarps * 32 - 1) / (kProducerWarps * 32);
template <int FMT> struct RawIQ;
template <> struct RawIQ<DG_IQ_C64> {
    float2 v[kPfPer];
    __device__ __forceinline__ void load(int e, const void *b, int i) { v[e] = __ldg(reinterpret_cast<const float2 *>(b) + i); }
    __device__ __forceinline__ void zero(int e) { v[e] = make_float2(0.f, 0.f); }
    __device__ __forceinline__ float2 get(int e) const { return v[e]; }
};
template <> struct RawIQ<DG_IQ_CI16> {
    int v[kPfPer];
    __device__ __forceinline__ void load(int e, const void *b, int i) { v[e] = __ldg(reinterpret_cast<const int *>(b) + i); }
    __device__ __forceinline__ void zero(int e) { v[e] = 0; }
    __device__ __forceinline__ float2 get(int e) const
    {
        return make_float2((float)(short)(v[e] & 0xffff), (float)(short)(v[e] >> 16));
    }
};
template <> struct RawIQ<DG_IQ_CI8> {
    short v[kPfPer];
    __device__ __forceinline__ void load(int e, const void *b, int i)
    {
        v[e] = (short)__ldg(reinterpret_cast<const unsigned short *>(b) + i);
    }
    __device__ __forceinline__ void zero(int e) { v[e] = 0; }
    __device__ __forceinline__ float2 get(int e) const
    {
        return make_float2((float)(signed char)(v[e] & 0xff), (float)(signed char)((v[e] >> 8) & 0xff));
    }
};

template <int FMT>
__device__ __forceinline__ void prefetch_windows(const TileInfo &t, int M, int w, RawIQ<FMT> &pf, int tid)
{
    const int SW = window_len(M);
    const int nb0 = t.bch * M + w * SW, L0 = t.Lmin + t.lb * kRows;
#pragma unroll
    for (int e = 0; e < kPfPer; ++e) {
        const int i = tid + kProducerWarps * 32 * e;
        int n = -1;
        const void *src = t.sd.y1;
        if (i < SW) n = nb0 + i;
        else if (i < 2 * SW + kRows) {
            n = nb0 + L0 + (i - SW);
            src = t.sd.y2;
        }
        if (n >= 0 && n < t.N) pf.load(e, src, n);
        else pf.zero(e);
    }
}

template <int FMT>
__device__ __forceinline__ void store_windows(const RawIQ<FMT> &pf, int M, float zs, float2 *sy1, float2 *sy2, int tid)
{
    const int SW = window_len(M);
#pragma unroll
    for (int e = 0; e < kPfPer; ++e) {
        const int i = tid + kProducerWarps * 32 * e;
        const float2 v = pf.get(e);
        if (i < SW) sy1[i] = make_float2(v.x * zs, v.y * zs);
        else if (i < 2 * SW + kRows) sy2[i - SW] = v;
    }
}

// Barrier of the producer warps (named barrier 1) that also ORs a flag over
// them: every producer gets the same answer, so they leave the tile loop
// together (no producer is left waiting at a later barrier).
__device__ __forceinline__ bool producers_sync_or(bool flag)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\t"
        "setp.ne.u32 pi, %1, 0;\n\t"
        "barrier.cta.red.or.pred po, 1, %2, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)flag), "r"(kProducerWarps * 32)
        : "memory");
    return r != 0;
}

template <int FMT, int DT, int P>
__global__ void __launch_bounds__(kWsThreads, 1)
    k_cdft_contract_tc(TcJob one, const TcJob *__restrict__ jobs, int njobs, const int *__restrict__ job_tiles,
                       unsigned wait_polls)
{
    constexpr int NA = ring_a<P>(), NB = ring_b<P>();
    constexpr int kSt = 2 * P * kBlockBytes;  // bytes of one stage's A (or B) blocks
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full_a[NA], empty_a[NA], full_b[NB], empty_b[NB], acc_full[2], acc_empty[2];
    __shared__ __align__(8) uint64_t drained;  // the MMA thread's last commit: all its MMAs are done
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    __shared__ SnapCache sc;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *sB0 = smem;
    float2 *sy1 = reinterpret_cast<float2 *>(smem + NB * kSt);
    float2 *sy2 = sy1 + kLagTileMaxChunk;
    // one job: its per-snapshot tables cached in shared memory; several
    // jobs: each tile is resolved to its job through job_tiles
    const bool multi = jobs != nullptr;
    if (!multi)
        for (int i = threadIdx.x; i <= one.S; i += blockDim.x) {
            sc.tbase[i] = one.tbase[i];
            sc.bbase[i] = one.bbase[i];
            if (i < one.S) {
                sc.lr[2 * i] = one.lr[2 * i];
                sc.lr[2 * i + 1] = one.lr[2 * i + 1];
                sc.layout[i] = one.layout[i];
                sc.sd[i] = one.sd[i];
            }
        }
    const JobTables single_tables{sc.tbase, sc.bbase, sc.lr, sc.layout, sc.sd};
    auto resolve = [&](int tile) -> TileInfo {
        if (!multi) return tile_info(single_tables, one.S, one.M, tile);
        int lo = 0, hi = njobs - 1;  // the job whose tile range holds the tile
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (job_tiles[mid] <= tile) lo = mid; else hi = mid - 1;
        }
        const TcJob &J = jobs[lo];
        const JobTables tb{J.tbase, J.bbase, J.lr, J.layout, J.sd};
        TileInfo t = tile_info(tb, J.S, J.M, tile - job_tiles[lo]);
        t.job = lo;
        return t;
    };
    auto job = [&](int j) -> const TcJob & { return multi ? jobs[j] : one; };
    if (threadIdx.x == 0) {
        for (int i = 0; i < NA; ++i) {
            mbar_init(smem_u32(&full_a[i]), kProducerWarps);
            mbar_init(smem_u32(&empty_a[i]), 1);
        }
        for (int i = 0; i < NB; ++i) {
            mbar_init(smem_u32(&full_b[i]), 1);
            mbar_init(smem_u32(&empty_b[i]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&acc_full[i]), 1);
            mbar_init(smem_u32(&acc_empty[i]), kEpilogueWarps);
        }
        mbar_init(smem_u32(&drained), 1);
        s_abort = 0;
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_slot), 512);
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_slot;
    const int ntiles = multi ? job_tiles[njobs] : sc.tbase[one.S];
    const int mine = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const uint32_t wl = wait_polls ? wait_polls : kWaitLimit;  // poll limit of the pipeline's waits

    if (warp < kProducerWarps) {
        // ---------------- producers: lane l of warp w forms row 32 (w % 4) + l
        // (a warp reaches only its quarter of the tensor-memory lanes), samples
        // 8 (w / 4) .. 8 (w / 4) + 7 of every 32-sample stage, and writes them
        // with tcgen05.st into the stage's A columns
        const int qd = warp & 3, sg = warp >> 2;
        const int row = 32 * qd + lane;
        const uint32_t tlane = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(kAccCols + 4 * sg);
        RawIQ<FMT> pf;
        bool have_pf = false;  // pf holds the window about to start
        bool stop = false;
        uint32_t g0 = 0;  // stages of the tiles before this one
        // A slot whose lag products are stored but not yet announced: its
        // tcgen05.st completes while the next stage is formed, and the
        // arrival on its full_a barrier follows then
        int pend = -1;
        auto announce = [&]() {
            if (pend >= 0) {
                tmem_wait_st();
                tc_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&full_a[pend]));
                pend = -1;
            }
        };
        for (int it = 0; it < mine && !stop; ++it) {
            const int tile = (int)blockIdx.x + it * (int)gridDim.x;
            const TileInfo t = resolve(tile);
            const int M = t.M, NJ = M / kKS;
            const int SWJ = window_len(M) / kKS;  // stages per window of a lag tile
            const float zs = job(t.job).zscale;
            const int *need = job(t.job).need;
            int pL = 0, pn0 = 0;
            bool pv = false;
            if (!t.lay) {
                const int64_t R = (int64_t)t.rNB * t.Bs;
                const int64_t g = (int64_t)t.rt * kRows + row;
                if (g < R) {
                    const int bl = t.rl0 + (int)(g / t.Bs);
                    pn0 = (int)(g % t.Bs) * M + 8 * sg;
                    pL = t.Lmin + bl;
                    pv = need[t.bb + bl] != 0;
                }
            }
            const int NW = t.lay ? NJ / SWJ : 1;          // windows of this tile
            const int JW = t.lay ? SWJ : NJ;              // stages per window
            for (int w = 0; w < NW; ++w) {
                // every producer is done with the previous window's shared
                // memory; all leave together on an abort (the only place a
                // producer leaves early, so all pass the same barriers)
                announce();
                if (producers_sync_or(s_abort != 0)) {
                    stop = true;
                    break;
                }
                if (t.lay) {
                    if (have_pf) store_windows<FMT>(pf, M, zs, sy1, sy2, threadIdx.x);
                    else stage_windows<FMT>(t, M, w, zs, sy1, sy2, threadIdx.x, kProducerWarps * 32);
                    asm volatile("bar.sync 1, %0;" ::"r"(kProducerWarps * 32) : "memory");
                }
                // the next window travels while this one's stages run: the
                // next of this tile, else the first of the next lag tile
                have_pf = false;
                if (t.lay && w + 1 < NW) {
                    prefetch_windows<FMT>(t, M, w + 1, pf, threadIdx.x);
                    have_pf = true;
                } else if (w + 1 == NW && it + 1 < mine) {
                    const TileInfo tn = resolve(tile + (int)gridDim.x);
                    if (tn.lay) {
                        prefetch_windows<FMT>(tn, tn.M, 0, pf, threadIdx.x);
                        have_pf = true;
                    }
                }
            for (int jw = 0; jw < JW; ++jw) {
                const int j = w * JW + jw;
                const uint32_t g = g0 + (uint32_t)j;
                const int slot = (int)(g % NA);
                // after an abort the remaining stages are skipped (no wait) up
                // to the next window's barrier
                if (s_abort) continue;
                if (g >= NA && !mbar_wait(smem_u32(&empty_a[slot]), ((g / NA) - 1) & 1u, wl)) {
                    s_abort = 1;
                    continue;
                }
                tc_after_sync();
                float2 x[8], y[8];
                if (t.lay) {
                    const int m0 = jw * kKS + 8 * sg;
#pragma unroll
                    for (int u = 0; u < 8; u += 2) {
                        const float4 q = *reinterpret_cast<const float4 *>(sy1 + m0 + u);
                        x[u] = make_float2(q.x, q.y);
                        x[u + 1] = make_float2(q.z, q.w);
                    }
                    const float2 *py = sy2 + m0 + row;
#pragma unroll
                    for (int u = 0; u < 8; ++u) y[u] = py[u];
                } else {
                    Raw<FMT> raw;
                    const int n = pn0 + j * kKS;
                    raw.fetch(t.sd.y1, t.sd.y2, n, n + pL, t.N, pv);
                    raw.decode(t.sd.y1, t.sd.y2, t.N, pv, x, y);
#pragma unroll
                    for (int u = 0; u < 8; ++u) x[u] = make_float2(x[u].x * zs, x[u].y * zs);
                }
                float zr[8], zi[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    zr[u] = fmaf(x[u].x, y[u].x, x[u].y * y[u].y);
                    zi[u] = fmaf(x[u].y, y[u].x, -x[u].x * y[u].y);
                }
                uint32_t hr[4], hi[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    hr[u] = pack2<DT>(zr[2 * u], zr[2 * u + 1]);
                    hi[u] = pack2<DT>(zi[2 * u], zi[2 * u + 1]);
                }
                announce();  // the previous stage's stores have had this stage's math to land
                const uint32_t ta = tlane + (uint32_t)(slot * a_stage_cols<P>());
                tmem_st4(ta, hr);       // high part, multiplies the re rows of B
                tmem_st4(ta + 16, hi);  // high part, im rows
                if (P == 2) {  // residuals z - high part, rounded to 16 bits
                    uint32_t lr[4], li[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float2 fr = unpack2<DT>(hr[u]), fi = unpack2<DT>(hi[u]);
                        lr[u] = pack2<DT>(zr[2 * u] - fr.x, zr[2 * u + 1] - fr.y);
                        li[u] = pack2<DT>(zi[2 * u] - fi.x, zi[2 * u + 1] - fi.y);
                    }
                    tmem_st4(ta + 32, lr);
                    tmem_st4(ta + 48, li);
                }
                pend = slot;
            }
            }
            g0 += (uint32_t)NJ;
        }
        announce();
    } else if (warp == kLoadWarp) {
        // ---------------- operand loader (one thread): B of every stage of
        // every tile, in order, into slot g % NB once the MMAs of stage
        // g - NB are done; it runs ahead of the MMAs by up to NB stages,
        // across tile boundaries
        if (lane == 0) {
            uint32_t issued = 0;  // stages whose copy has been issued
            uint32_t g0 = 0;
            for (int it = 0; it < mine && !s_abort; ++it) {
                const TileInfo t = resolve((int)blockIdx.x + it * (int)gridDim.x);
                const int NJ = t.M / kKS;
                const unsigned char *bsrc =
                    reinterpret_cast<const unsigned char *>(job(t.job).btab) + (size_t)t.s * NJ * kSt;
                for (int j = 0; j < NJ; ++j) {
                    const uint32_t g = g0 + (uint32_t)j;
                    const int slot = (int)(g % NB);
                    if ((g >= NB && !mbar_wait(smem_u32(&empty_b[slot]), ((g / NB) - 1) & 1u, wl)) || s_abort) {
                        s_abort = 1;
                        break;
                    }
                    mbar_expect_tx(smem_u32(&full_b[slot]), kSt);
                    bulk_g2s(smem_u32(sB0 + slot * kSt), bsrc + (size_t)j * kSt, kSt, smem_u32(&full_b[slot]));
                    issued = g + 1;
                }
                g0 += (uint32_t)NJ;
            }
            // after an abort, the copies still in flight (at most the last NB
            // issued) land before the CTA leaves: shared memory is not
            // released under a bulk copy
            if (s_abort)
                for (uint32_t g = issued > (uint32_t)NB ? issued - NB : 0; g < issued; ++g)
                    mbar_wait(smem_u32(&full_b[g % NB]), (g / NB) & 1u);
        }
    } else if (warp == kMmaWarp) {
        // ---------------- MMA thread: waits for A and B of each stage,
        // issues its MMAs and commits them to the stage's empty barriers; it
        // waits on MMA completion only to reuse an accumulator
        if (lane == 0) {
            const uint32_t id = idesc<DT>();
            bool alive = true;
            uint32_t g0 = 0;
            for (int it = 0; it < mine && alive && !s_abort; ++it) {
                const int NJ = (multi ? resolve((int)blockIdx.x + it * (int)gridDim.x).M : one.M) / kKS;
                // the accumulator of this tile was drained (tile it - 2)
                const int acc = it & 1;
                if (it >= 2 && !mbar_wait(smem_u32(&acc_empty[acc]), ((uint32_t)(it / 2) - 1) & 1u, wl)) {
                    alive = false;
                    break;
                }
                tc_after_sync();
                const uint32_t dtm = tmem + (uint32_t)(128 * acc);
                for (int j = 0; j < NJ; ++j) {
                    const uint32_t g = g0 + (uint32_t)j;
                    const int sa = (int)(g % NA), sb = (int)(g % NB);
                    if (!mbar_wait(smem_u32(&full_a[sa]), (g / NA) & 1u, wl) ||
                        !mbar_wait(smem_u32(&full_b[sb]), (g / NB) & 1u, wl) || s_abort) {
                        alive = false;
                        break;
                    }
                    tc_after_sync();
                    const uint32_t at0 = tmem + (uint32_t)(kAccCols + sa * a_stage_cols<P>());
                    const unsigned char *sB = sB0 + sb * kSt;
                    constexpr int NPROD = P == 2 ? 3 : 1;
#pragma unroll
                    for (int blk = 0; blk < 2; ++blk)
#pragma unroll
                        for (int kk = 0; kk < kKS; kk += 16)
#pragma unroll
                            for (int pr = 0; pr < NPROD; ++pr) {
                                const int pa = pr == 1 ? 1 : 0, pb = pr == 2 ? 1 : 0;
                                const uint32_t at = at0 + (uint32_t)((2 * pa + blk) * 16 + kk / 2);
                                const uint64_t bd = sdesc(smem_u32(sB + (2 * pb + blk) * kBlockBytes) + kk * 16);
                                mma_f16_ta(dtm, at, bd, id, (j > 0 || blk > 0 || kk > 0 || pr > 0) ? 1u : 0u);
                            }
                    mma_commit(smem_u32(&empty_a[sa]));
                    mma_commit(smem_u32(&empty_b[sb]));
                    if (j == NJ - 1) mma_commit(smem_u32(&acc_full[acc]));  // the tile's accumulator is final
                }
                g0 += (uint32_t)NJ;
            }
            if (!alive) s_abort = 1;
            // completes once every MMA this thread issued is done
            mma_commit(smem_u32(&drained));
        }
    } else {
        // ---------------- drain finished accumulators: the last four warps
        const int q = warp & 3;
        for (int it = 1; it <= mine && !s_abort; ++it) {
            // drain tile it - 1
            const int d = it - 1, acc = d & 1;
            if (!mbar_wait(smem_u32(&acc_full[acc]), (uint32_t)(d / 2) & 1u, wl)) {
                s_abort = 1;
                break;
            }
            tc_after_sync();
            const TileInfo t = resolve((int)blockIdx.x + d * (int)gridDim.x);
            const TcJob &J = job(t.job);
            const int *need = J.need;
            const int Bmax = J.Bmax;
            float *W = J.W;
            const int row = 32 * q + lane;
            bool valid;
            int64_t wrow;
            if (t.lay) {
                const int bl = t.lb * kRows + row;
                valid = bl < t.NB && need[t.bb + bl] != 0;
                wrow = ((int64_t)(t.bb + bl) * Bmax + t.bch) * 128;
            } else {
                const int64_t g = (int64_t)t.rt * kRows + row;
                valid = g < (int64_t)t.rNB * t.Bs;
                const int bl = valid ? t.rl0 + (int)(g / t.Bs) : 0;
                valid = valid && need[t.bb + bl] != 0;
                wrow = ((int64_t)(t.bb + bl) * Bmax + (valid ? g % t.Bs : 0)) * 128;
            }
            const float inv = 1.0f / J.zscale;
            const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(128 * acc);
#pragma unroll 1
            for (int c = 0; c < 128; c += 32) {
                uint32_t r[32];
                tmem_ld32(tb + (uint32_t)c, r);
                if (valid) {
                    float4 *w = reinterpret_cast<float4 *>(W + wrow + c);
#pragma unroll
                    for (int v = 0; v < 8; ++v)
                        w[v] = make_float4(__uint_as_float(r[4 * v]) * inv, __uint_as_float(r[4 * v + 1]) * inv,
                                           __uint_as_float(r[4 * v + 2]) * inv, __uint_as_float(r[4 * v + 3]) * inv);
                }
            }
            tc_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acc_empty[acc]));
        }
    }
    __syncthreads();
    // after an abort, every MMA issued must complete before TMEM is freed
    if (s_abort && threadIdx.x == 0) {
        mbar_wait(smem_u32(&drained), 0u);
        if (multi)  // every job's surface is incomplete
            for (int j = 0; j < njobs; ++j) atomicOr(jobs[j].err, ERR_TIMEOUT);
        else
            atomicOr(one.err, ERR_TIMEOUT);
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------
// Hankel tiles: 512 consecutive lags L0 .. L0 + 511 of snapshot s at chunk b.
// The contraction is regrouped so that the lag-dependent operand is the raw
// capture:
//     W_b(L, q) = sum_m G_q[m] conj(y2[bM + m + L]),  G_q[m] = y1[bM + m] e^{j 2 pi nu_q m}.
// A (128 x 2M, K-major, formed per 32-sample stage by the producers): row q
// holds [G_re | G_im] and row 64 + q holds [G_im | -G_re] over the K halves
// (re, im of y2), so that D = A B^T gives the real (rows < 64) and imaginary
// (rows >= 64) parts of W in the planar order of W's rows.
// B (N x 2M): y2 read as a Hankel matrix. The tile's lags are split into 8
// phases L0 + r + 8n (n < 64); for phase r, element (n, k) of the real half
// is y2_re[bM + L0 + r + 8n + k], which is element 8n + k of the window copy
// shifted by r. In the canonical no-swizzle K-major layout a core matrix
// (8 rows x 8 elements) of rows 8g .. 8g + 7 and elements 8h .. 8h + 7 is then
// the 64 consecutive window elements from 64g + 8h: K-adjacent core matrices
// are 16 B apart (leading byte offset) and 8-row groups 128 B apart (stride
// byte offset), and the window copies are all the B operand there is. Each
// phase is one MMA of N = 64 into its own 64 accumulator columns; the one
// accumulator (512 columns) is drained by the epilogue before the next
// tile's first MMA. The window copies (8 phases x re, im x high, residual)
// stay in shared memory for the whole tile; the producers rebuild them for
// the next tile once the MMAs of the previous tile have completed (acc_full).
// ---------------------------------------------------------------------------
constexpr int kHkPhases = 8;
constexpr int kHkN = kHkLags / kHkPhases;                 // MMA N: lags per phase
constexpr int kHkWin = kLagTileMaxChunk + kHkLags;        // elements of one window copy (>= M + 8 * 31)
constexpr int kHkPlane = kHkWin * 2;                      // bytes of one 16-bit copy
constexpr int kHkEpiWarp0 = kProducerWarps + 1;           // producers, the MMA warp, then 4 epilogue warps
constexpr int kHkThreads = (kProducerWarps + 1 + kEpilogueWarps) * 32;
template <int P> __host__ __device__ constexpr int hk_ring() { return P == 2 ? 3 : 4; }
template <int P> __host__ __device__ constexpr int hk_smem_bytes()
{
    return hk_ring<P>() * (2 * P * kBlockBytes) + kHkPhases * 2 * P * kHkPlane +
           (kLagTileMaxChunk + kHkWin + 8) * (int)sizeof(float2);
}

// B descriptor of a Hankel view: leading byte offset 16, stride byte offset 128.
__device__ __forceinline__ uint64_t hdesc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(16 >> 4) << 16) | ((uint64_t)(128 >> 4) << 32) |
           (1ull << 46);
}

template <int DT> __device__ __forceinline__ uint32_t idesc_hk()
{
    const uint32_t t = DT == DG_CONTRACT_BF16 ? 1u : 0u;
    return (1u << 4) | (t << 7) | (t << 10) | ((uint32_t)(kHkN >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

struct HkCache {  // per-snapshot tables of the batch, in shared memory
    int hbase[kSnapCache + 1];
    int bbase[kSnapCache + 1];
    int lr[2 * kSnapCache];
    float nubase[kSnapCache], delta[kSnapCache];
    StepDesc sd[kSnapCache];
};

struct HkTile {
    int s, lb, bch, NB, N, Lmin, bb;
    StepDesc sd;
};

__device__ __forceinline__ HkTile hk_tile(const HkCache &c, int S, int tile)
{
    HkTile t;
    t.s = step_of_tile(c.hbase, S, tile);
    const int lt = tile - c.hbase[t.s];
    t.sd = c.sd[t.s];
    t.N = t.sd.n;
    const int lo = c.lr[2 * t.s], hi = c.lr[2 * t.s + 1];
    t.NB = hi >= lo ? hi - lo + 1 : 0;
    if (t.NB > c.bbase[t.s + 1] - c.bbase[t.s]) t.NB = 0;  // as the planner: no tiles then
    const int NLB = max((t.NB + kHkLags - 1) / kHkLags, 1);
    t.lb = lt % NLB;
    t.bch = lt / NLB;
    t.Lmin = lo;
    t.bb = c.bbase[t.s];
    return t;
}

template <int FMT, int DT, int P>
__global__ void __launch_bounds__(kHkThreads, 1) k_cdft_contract_hk(CdftBatch a)
{
    constexpr int NA = hk_ring<P>();
    constexpr int kSt = 2 * P * kBlockBytes;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full_a[NA], empty_a[NA], acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    __shared__ HkCache sc;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *sA0 = smem;
    unsigned char *sW = smem + NA * kSt;  // window copies [phase][part][re, im] of kHkPlane bytes
    float2 *sy1 = reinterpret_cast<float2 *>(sW + kHkPhases * 2 * P * kHkPlane);
    float2 *sy2 = sy1 + kLagTileMaxChunk;  // kHkWin + 8 samples
    const int M = a.M, NJ = M / kKS, S = a.S;

    for (int i = threadIdx.x; i <= S; i += blockDim.x) {
        sc.hbase[i] = a.hbase[i];
        sc.bbase[i] = a.bbase[i];
        if (i < S) {
            sc.lr[2 * i] = a.lr[2 * i];
            sc.lr[2 * i + 1] = a.lr[2 * i + 1];
            sc.nubase[i] = a.nubase[i];
            sc.delta[i] = a.delta[i];
            sc.sd[i] = a.sd[i];
        }
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < NA; ++i) {
            mbar_init(smem_u32(&full_a[i]), kProducerWarps);
            mbar_init(smem_u32(&empty_a[i]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&acc_full[i]), 1);
            mbar_init(smem_u32(&acc_empty[i]), kEpilogueWarps);
        }
        s_abort = 0;
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_slot), kHkLags);
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_slot;
    const int ntiles = sc.hbase[S];
    const int mine = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const float zs = sqrtf(a.zscale);  // on y1 and on y2: their product carries zscale

    if (warp < kProducerWarps) {
        // ---------------- producers
        const int part = warp >> 3, qset = warp & 7;
        const int rin = lane & 7, kg = lane >> 3;
        const int q = 8 * qset + rin;
        const int ptid = threadIdx.x, pthreads = kProducerWarps * 32;
        for (int it = 0; it < mine; ++it) {
            // the window copies are free once the previous tile's MMAs have
            // completed; all producers leave together on an abort
            bool fail = false;
            if (ptid == 0 && it >= 1) fail = !mbar_wait(smem_u32(&acc_full[0]), (uint32_t)(it - 1) & 1u);
            if (producers_sync_or(fail || s_abort != 0)) {
                s_abort = 1;
                break;
            }
            const int tile = (int)blockIdx.x + it * (int)gridDim.x;
            const HkTile t = hk_tile(sc, S, tile);
            const int nb0 = t.bch * M, L0 = t.Lmin + t.lb * kHkLags;
            for (int i = ptid; i < M; i += pthreads) {
                const int n = nb0 + i;
                const float2 v = n < t.N ? IQ<FMT>::load(t.sd.y1, n) : make_float2(0.f, 0.f);
                sy1[i] = make_float2(v.x * zs, v.y * zs);
            }
            for (int i = ptid; i < kHkWin + 8; i += pthreads) {
                const int n2 = nb0 + L0 + i;
                const float2 v = (n2 >= 0 && n2 < t.N) ? IQ<FMT>::load(t.sd.y2, n2) : make_float2(0.f, 0.f);
                sy2[i] = make_float2(v.x * zs, v.y * zs);
            }
            asm volatile("bar.sync 1, %0;" ::"r"(kProducerWarps * 32) : "memory");
            // window copies: copy r element e = y2 window sample r + e, 8 elements per task
            for (int task = ptid; task < kHkPhases * (kHkWin / 8); task += pthreads) {
                const int r = task / (kHkWin / 8), e0 = 8 * (task % (kHkWin / 8));
                float vr[8], vi[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float2 v = sy2[r + e0 + u];
                    vr[u] = v.x;
                    vi[u] = v.y;
                }
                uint32_t hr[4], hi[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    hr[u] = pack2<DT>(vr[2 * u], vr[2 * u + 1]);
                    hi[u] = pack2<DT>(vi[2 * u], vi[2 * u + 1]);
                }
                unsigned char *base = sW + (size_t)r * 2 * P * kHkPlane + 2 * e0;
                *reinterpret_cast<uint4 *>(base) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
                *reinterpret_cast<uint4 *>(base + kHkPlane) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                if (P == 2) {
                    uint32_t lr[4], li[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float2 fr = unpack2<DT>(hr[u]), fi = unpack2<DT>(hi[u]);
                        lr[u] = pack2<DT>(vr[2 * u] - fr.x, vr[2 * u + 1] - fr.y);
                        li[u] = pack2<DT>(vi[2 * u] - fi.x, vi[2 * u + 1] - fi.y);
                    }
                    *reinterpret_cast<uint4 *>(base + 2 * kHkPlane) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
                    *reinterpret_cast<uint4 *>(base + 3 * kHkPlane) = make_uint4(li[0], li[1], li[2], li[3]);
                }
            }
            // A of every stage: G_q[m] = y1[m] e^{j 2 pi nu_q m} (the bin
            // frequency in FP32 and the phase of sample m from the exact
            // product split, as the DFT tables form them)
            const float nuq = fmaf((float)q, sc.delta[t.s], sc.nubase[t.s]);
            const uint32_t g0 = (uint32_t)it * (uint32_t)NJ;
            for (int j = 0; j < NJ; ++j) {
                const uint32_t g = g0 + (uint32_t)j;
                const int slot = (int)(g % NA);
                if (g >= NA && !mbar_wait(smem_u32(&empty_a[slot]), ((g / NA) - 1) & 1u)) s_abort = 1;
                if (s_abort) break;
                unsigned char *sA = sA0 + slot * kSt;
                const int m0 = j * kKS + 8 * kg;
                float gv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float2 x = sy1[m0 + u];
                    float sn, cs;
                    sincospif(2.0f * frac_mul(nuq, (float)(m0 + u)), &sn, &cs);
                    gv[u] = part == 0 ? fmaf(x.x, cs, -x.y * sn) : fmaf(x.x, sn, x.y * cs);
                }
                // part 0 (G_re): row q of the y2_re half, row 64 + q of the y2_im half (negated);
                // part 1 (G_im): row 64 + q of the y2_re half, row q of the y2_im half
                const int row0 = part == 0 ? q : 64 + q, row1 = part == 0 ? 64 + q : q;
                const float sg = part == 0 ? -1.f : 1.f;
                uint32_t h0[4], h1[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    h0[u] = pack2<DT>(gv[2 * u], gv[2 * u + 1]);
                    h1[u] = pack2<DT>(sg * gv[2 * u], sg * gv[2 * u + 1]);
                }
                *reinterpret_cast<uint4 *>(sA + blk_off(row0, 8 * kg)) = make_uint4(h0[0], h0[1], h0[2], h0[3]);
                *reinterpret_cast<uint4 *>(sA + kBlockBytes + blk_off(row1, 8 * kg)) =
                    make_uint4(h1[0], h1[1], h1[2], h1[3]);
                if (P == 2) {
                    uint32_t l0[4], l1[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float2 f0 = unpack2<DT>(h0[u]), f1 = unpack2<DT>(h1[u]);
                        l0[u] = pack2<DT>(gv[2 * u] - f0.x, gv[2 * u + 1] - f0.y);
                        l1[u] = pack2<DT>(sg * gv[2 * u] - f1.x, sg * gv[2 * u + 1] - f1.y);
                    }
                    *reinterpret_cast<uint4 *>(sA + 2 * kBlockBytes + blk_off(row0, 8 * kg)) =
                        make_uint4(l0[0], l0[1], l0[2], l0[3]);
                    *reinterpret_cast<uint4 *>(sA + 3 * kBlockBytes + blk_off(row1, 8 * kg)) =
                        make_uint4(l1[0], l1[1], l1[2], l1[3]);
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&full_a[slot]));
            }
        }
    } else if (warp == kMmaWarp) {
        // ---------------- MMA thread: one accumulator of kHkLags columns;
        // descriptors are formed by adding byte offsets >> 4 to base
        // descriptors (the start field cannot carry: shared memory < 256 KB)
        if (lane == 0) {
            const uint32_t id = idesc_hk<DT>();
            const uint64_t a0 = sdesc(smem_u32(sA0)), w0 = hdesc(smem_u32(sW));
            bool alive = true;
            for (int it = 0; it < mine && alive && !s_abort; ++it) {
                const uint32_t g0 = (uint32_t)it * (uint32_t)NJ;
                // the accumulator was drained (tile it - 1)
                if (it >= 1 && !mbar_wait(smem_u32(&acc_empty[0]), ((uint32_t)(it - 1)) & 1u)) {
                    alive = false;
                    break;
                }
                tc_after_sync();
                for (int j = 0; j < NJ; ++j) {
                    const uint32_t g = g0 + (uint32_t)j;
                    const int sa = (int)(g % NA);
                    if (!mbar_wait(smem_u32(&full_a[sa]), (g / NA) & 1u) || s_abort) {
                        alive = false;
                        break;
                    }
                    tc_after_sync();
                    const uint64_t as = a0 + (uint64_t)((sa * kSt) >> 4);
                    const uint64_t ws = w0 + (uint64_t)((2 * j * kKS) >> 4);
                    constexpr int NPROD = P == 2 ? 3 : 1;
#pragma unroll
                    for (int blk = 0; blk < 2; ++blk)
#pragma unroll
                        for (int kk = 0; kk < kKS; kk += 16)
#pragma unroll
                            for (int pr = 0; pr < NPROD; ++pr) {
                                const int pa = pr == 1 ? 1 : 0, pb = pr == 2 ? 1 : 0;
                                const uint64_t ad = as + (uint64_t)(((2 * pa + blk) * kBlockBytes + kk * 16) >> 4);
                                const uint64_t bd = ws + (uint64_t)(((2 * pb + blk) * kHkPlane + 2 * kk) >> 4);
                                const uint32_t accf = (j > 0 || blk > 0 || kk > 0 || pr > 0) ? 1u : 0u;
#pragma unroll
                                for (int r = 0; r < kHkPhases; ++r)
                                    mma_f16(tmem + (uint32_t)(kHkN * r), ad,
                                            bd + (uint64_t)((r * 2 * P * kHkPlane) >> 4), id, accf);
                            }
                    mma_commit(smem_u32(&empty_a[sa]));
                    if (j == NJ - 1) mma_commit(smem_u32(&acc_full[0]));
                }
            }
            if (!alive) s_abort = 1;
        }
    } else {
        // ---------------- drain finished accumulators: the last four warps
        const int qw = warp & 3;
        for (int it = 1; it <= mine && !s_abort; ++it) {
            const int d = it - 1;
            if (!mbar_wait(smem_u32(&acc_full[0]), (uint32_t)d & 1u)) {
                s_abort = 1;
                break;
            }
            tc_after_sync();
            const HkTile t = hk_tile(sc, S, (int)blockIdx.x + d * (int)gridDim.x);
            const int row = 32 * qw + lane;
            const float inv = 1.0f / a.zscale;
            const uint32_t tb = tmem + ((uint32_t)(32 * qw) << 16);
#pragma unroll 1
            for (int c0 = 0; c0 < kHkLags; c0 += 32) {  // 32 columns of phase c0 / kHkN at a time
                uint32_t v[32];
                tmem_ld32(tb + (uint32_t)c0, v);
                const int r = c0 / kHkN, nb = c0 % kHkN;
#pragma unroll 4
                for (int u = 0; u < 32; ++u) {
                    const int bl = t.lb * kHkLags + r + 8 * (nb + u);
                    if (bl < t.NB && a.need[t.bb + bl] != 0)
                        a.W[((int64_t)(t.bb + bl) * a.Bmax + t.bch) * 128 + row] = __uint_as_float(v[u]) * inv;
                }
            }
            tc_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acc_empty[0]));
        }
    }
    __syncthreads();
    if (s_abort && mine > 0 && threadIdx.x == 0) {
        mbar_wait(smem_u32(&acc_full[0]), (uint32_t)(mine - 1) & 1u);
        atomicOr(a.err, ERR_TIMEOUT);
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 0) tmem_dealloc(tmem, kHkLags);
}

cudaError_t launch_cdft_btab(const CdftBatch &a, int mode, void *btab, cudaStream_t st)
{
    const size_t n = (size_t)(a.M / kKS) * 64 * (kKS / 8);
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
static cudaError_t launch_mma(const TcJob &one, const TcJob *jobs, int njobs, const int *job_tiles, int grid,
                              unsigned wait_polls, cudaStream_t st)
{
    // lag tiles stage windows of kLagTileMaxChunk + 128 samples
    const int smem = tc_smem_bytes<P>();
    cudaError_t e = cudaFuncSetAttribute(k_cdft_contract_tc<FMT, DT, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_cdft_contract_tc<FMT, DT, P><<<(unsigned)grid, kWsThreads, smem, st>>>(one, jobs, njobs, job_tiles, wait_polls);
    return cudaGetLastError();
}

template <int FMT, int DT, int P>
static cudaError_t launch_hk(const CdftBatch &a, int grid, cudaStream_t st)
{
    const int smem = hk_smem_bytes<P>();
    cudaError_t e = cudaFuncSetAttribute(k_cdft_contract_hk<FMT, DT, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_cdft_contract_hk<FMT, DT, P><<<(unsigned)grid, kHkThreads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int DT, int P>
static cudaError_t launch_hk_fmt(const CdftBatch &a, int grid, int fmt, cudaStream_t st)
{
    switch (fmt) {
    case DG_IQ_C64: return launch_hk<DG_IQ_C64, DT, P>(a, grid, st);
    case DG_IQ_CI16: return launch_hk<DG_IQ_CI16, DT, P>(a, grid, st);
    default: return launch_hk<DG_IQ_CI8, DT, P>(a, grid, st);
    }
}

template <int DT, int P>
static cudaError_t launch_fmt(const TcJob &one, const TcJob *jobs, int njobs, const int *job_tiles, int grid,
                              unsigned wait_polls, int fmt, cudaStream_t st)
{
    switch (fmt) {
    case DG_IQ_C64: return launch_mma<DG_IQ_C64, DT, P>(one, jobs, njobs, job_tiles, grid, wait_polls, st);
    case DG_IQ_CI16: return launch_mma<DG_IQ_CI16, DT, P>(one, jobs, njobs, job_tiles, grid, wait_polls, st);
    default: return launch_mma<DG_IQ_CI8, DT, P>(one, jobs, njobs, job_tiles, grid, wait_polls, st);
    }
}

static cudaError_t launch_mode(const TcJob &one, const TcJob *jobs, int njobs, const int *job_tiles, int grid,
                               unsigned wait_polls, int fmt, int mode, cudaStream_t st)
{
    switch (mode) {
    case DG_CONTRACT_BF16: return launch_fmt<DG_CONTRACT_BF16, 1>(one, jobs, njobs, job_tiles, grid, wait_polls, fmt, st);
    case DG_CONTRACT_FP16: return launch_fmt<DG_CONTRACT_FP16, 1>(one, jobs, njobs, job_tiles, grid, wait_polls, fmt, st);
    case DG_CONTRACT_BF16X3: return launch_fmt<DG_CONTRACT_BF16, 2>(one, jobs, njobs, job_tiles, grid, wait_polls, fmt, st);
    default: return launch_fmt<DG_CONTRACT_FP16, 2>(one, jobs, njobs, job_tiles, grid, wait_polls, fmt, st);
    }
}

TcJob tc_job(const CdftBatch &a, const void *btab)
{
    TcJob j;
    j.sd = a.sd;
    j.tbase = a.tbase;
    j.bbase = a.bbase;
    j.lr = a.lr;
    j.layout = a.layout;
    j.need = a.need;
    j.W = a.W;
    j.btab = btab;
    j.err = a.err;
    j.S = a.S;
    j.M = a.M;
    j.Bmax = a.Bmax;
    j.zscale = a.zscale;
    return j;
}

cudaError_t launch_cdft_contract_mma(const CdftBatch &a, int grid, int fmt, int mode, cudaStream_t st)
{
    return launch_mode(tc_job(a, a.btab), nullptr, 0, nullptr, grid, a.wait_polls, fmt, mode, st);
}

cudaError_t launch_cdft_contract_jobs(const TcJob *jobs, int n, const int *job_tiles, int grid, int fmt, int mode,
                                      unsigned wait_polls, cudaStream_t st)
{
    TcJob none{};
    return launch_mode(none, jobs, n, job_tiles, grid, wait_polls, fmt, mode, st);
}

__global__ void k_tc_job_tiles(const TcJob *jobs, int n, int *job_tiles)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int run = 0;
    for (int j = 0; j < n; ++j) {
        job_tiles[j] = run;
        run += jobs[j].tbase[jobs[j].S];
    }
    job_tiles[n] = run;
}

cudaError_t launch_tc_job_tiles(const TcJob *jobs, int n, int *job_tiles, cudaStream_t st)
{
    k_tc_job_tiles<<<1, 32, 0, st>>>(jobs, n, job_tiles);
    return cudaGetLastError();
}

cudaError_t launch_cdft_contract_hankel(const CdftBatch &a, int grid, int fmt, int mode, cudaStream_t st)
{
    switch (mode) {
    case DG_CONTRACT_BF16: return launch_hk_fmt<DG_CONTRACT_BF16, 1>(a, grid, fmt, st);
    case DG_CONTRACT_FP16: return launch_hk_fmt<DG_CONTRACT_FP16, 1>(a, grid, fmt, st);
    case DG_CONTRACT_BF16X3: return launch_hk_fmt<DG_CONTRACT_BF16, 2>(a, grid, fmt, st);
    default: return launch_hk_fmt<DG_CONTRACT_FP16, 2>(a, grid, fmt, st);
    }
}

}  // namespace dg
