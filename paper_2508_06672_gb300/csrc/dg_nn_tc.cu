// dg_nn_tc.cu -- the proposal network's 3 x 3 convolutions on the tensor
// cores (tcgen05, sm_103a): BF16 activations and weights, FP32 accumulation.
//
// Both are implicit GEMMs with the accumulator in tensor memory and the
// operands in shared memory (no swizzle, K-major canonical layout: 8-row x
// 16-byte core matrices):
//
//   forward / data gradient: rows = 128 consecutive pixels of one image
//     row (two image rows per CTA, one accumulator each), columns = output
//     channels, K = (input channel, tap) pairs:
//       y[n,o,i,j] = b[o] + sum_{c,u,v} w[o,c,u,v] x[n,c,i+u-1,j+v-1]
//     The data gradient is the same product with dy as the input, the
//     weights transposed (input and output channels swapped) and the taps
//     flipped:
//       dx[n,c,i,j] = sum_{o,u,v} w[o,c,u,v] dy[n,o,i-u+1,j-v+1]
//     The input rows a CTA needs are staged once per block of 32 channels;
//     each tap's A operand is that staging seen through a shifted
//     descriptor (k_conv3x3_tc). The weights are converted to BF16 blocks
//     once per call and stream in by bulk copy.
//   weight gradient: rows = output channels, columns = (input channel, tap)
//     pairs plus one column of ones (the bias gradient), K = pixels:
//       dw[o,c,u,v] = sum_{n,i,j} dy[n,o,i,j] x[n,c,i+u-1,j+v-1]
//       db[o]       = sum_{n,i,j} dy[n,o,i,j]
//     split over pixel ranges; the partial sums are added in a fixed order.
//     128 threads gather a 32-pixel K block of both operands (rounded to
//     BF16) into one of two shared-memory stages while one thread issues the
//     MMAs of the previous block.
// The FP32 kernels in dg_nn.cu stay as the reference.
#include <cuda_bf16.h>

#include <algorithm>

#include "dg_internal.cuh"

namespace dg {
namespace {

constexpr int kRowsTc = 128;                 // MMA M
constexpr int kKB = 32;                      // K elements per staged block
constexpr int kABytes = kRowsTc * kKB * 2;   // one 128 x 32 BF16 block
constexpr uint32_t kNnWaitLimit = 1u << 24;  // polls before an mbarrier wait gives up

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) in a K-major block of 32 K elements
__device__ __forceinline__ uint32_t kmaj(int row, int k)
{
    return (uint32_t)(((row >> 3) * 4 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// shared-memory descriptor: start >> 4, leading byte offset 128 (K-adjacent
// core matrices), stride byte offset 512 (8-row groups), version 1, no swizzle
__device__ __forceinline__ uint64_t nn_sdesc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) |
           (1ull << 46);
}

// instruction descriptor, kind::f16: FP32 D, BF16 A and B, both K-major,
// N >> 3 at [17, 23), M >> 4 at [24, 29)
__device__ __forceinline__ uint32_t nn_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kRowsTc >> 4) << 24);
}

__device__ __forceinline__ void nn_mma(uint32_t d, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(ad), "l"(bd), "r"(id), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void nn_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void nn_mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// bounded wait on an mbarrier phase: false after 2 s of the global timer
// (checked every 256 polls) or kNnWaitLimit polls
__device__ __forceinline__ bool nn_wait(uint32_t bar, uint32_t parity)
{
    uint64_t t0 = 0;
    for (uint32_t i = 0; i < kNnWaitLimit; ++i) {
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
            uint64_t now;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
            if (t0 == 0) t0 = now;
            else if (now - t0 > 2000000000ull) return false;
        }
    }
    return false;
}

__device__ __forceinline__ void nn_tmem_alloc(uint32_t slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void nn_tmem_free(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void nn_ld32(uint32_t taddr, uint32_t (&r)[32])
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

__device__ __forceinline__ void nn_fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void nn_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void nn_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ uint16_t bf16_bits(float v)
{
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    return *reinterpret_cast<const uint16_t *>(&h);
}

// Tensor-memory columns of an accumulator of n columns (a power of two >= 32).
__host__ __device__ constexpr int tmem_cols(int n) { return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : 256; }

}  // namespace

// ---------------------------------------------------------------------------
// Forward and data gradient: halo-staged implicit GEMM. A CTA computes
// kHaloRows output rows x 128 pixels (j0 .. j0 + 127) of image n for output
// channels o0 .. o0 + NT - 1 (NT a multiple of 16, <= 128). K runs over
// (channel block of 32, tap): for each channel block the CTA stages the
// kHaloRows + 2 input rows it needs, pixels j0 - 1 .. j0 + 128, as BF16 in
// shared memory, one 16-byte row per (input row, 8 channels, pixel). In the
// canonical K-major layout a core matrix is then 8 consecutive pixels of one
// 8-channel group, the 8-pixel groups 128 B apart and the channel groups
// kHaloQ * 16 B apart, so the A operand of tap (u, v) for output row r is the
// same staging seen from input row r + u and shifted by v pixels: a
// different descriptor start, nothing gathered per tap. The weights come
// pre-converted (k_conv_tc_wimg: one 32-channel x NT block per (channel
// block, tap) in the canonical layout) and stream through a ring of
// kWRing shared-memory slots by bulk copy. One thread issues the MMAs of a
// channel block (9 taps x kHaloRows rows x 2 K-steps of 16) while every
// thread stages the next block's input rows into the other buffer.
// x: [B][CI][H][W]; y: [B][CO][H][W]; b may be NULL.
// ---------------------------------------------------------------------------
constexpr int kHaloRows = 2;                                   // output rows per CTA
constexpr int kHaloCB = 32;                                    // input channels per block
constexpr int kHaloQ = kRowsTc + 2;                            // staged pixels per input row
constexpr int kHaloBytes = (kHaloRows + 2) * (kHaloCB / 8) * kHaloQ * 16;
constexpr int kWRing = 5;                                      // weight blocks in shared memory
constexpr int kConvThreads = 256;

// accumulator columns of one output row (NT rounded up to the 32-column loads)
__host__ __device__ constexpr int acc_stride(int nt) { return (nt + 31) / 32 * 32; }

__host__ __device__ constexpr int conv_tc_smem(int nt) { return 2 * kHaloBytes + kWRing * nt * kHaloCB * 2; }

// elements (16-bit) of the pre-converted weights of a layer with CI inputs and CO outputs
__host__ __device__ inline int64_t wimg_elems(int ci, int co, int nt)
{
    return (int64_t)((co + nt - 1) / nt) * ((ci + kHaloCB - 1) / kHaloCB) * 9 * nt * kHaloCB;
}

// shared-memory descriptor of staged input rows: K-adjacent core matrices
// (8-channel groups) kHaloQ * 16 B apart, 8-pixel groups 128 B apart
__device__ __forceinline__ uint64_t halo_desc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((kHaloQ * 16) >> 4) << 16) |
           ((uint64_t)(128 >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void nn_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void nn_bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Weights of the forward convolution (TR = false: w [CO][CI][3][3]) or of the
// data gradient (TR = true: the forward's w [CI][CO][3][3], transposed, taps
// flipped) as BF16 blocks: block (output block ob, channel block cb, tap) =
// NT output channels x 32 input channels in the canonical K-major layout
// (kmaj), zeros past CO and CI.
template <bool TR>
__global__ void k_conv_tc_wimg(const float *__restrict__ w, uint16_t *__restrict__ wimg, int CI, int CO, int NT)
{
    const int ncb = (CI + kHaloCB - 1) / kHaloCB, ob = (CO + NT - 1) / NT;
    const int64_t items = (int64_t)ob * ncb * 9 * NT * (kHaloCB / 8);
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < items;
         it += (int64_t)gridDim.x * blockDim.x) {
        const int kg = (int)(it % (kHaloCB / 8));
        const int ol = (int)((it / (kHaloCB / 8)) % NT);
        const int64_t blk = it / ((kHaloCB / 8) * NT);
        const int tap = (int)(blk % 9), cb = (int)((blk / 9) % ncb), obi = (int)(blk / (9 * ncb));
        const int o = obi * NT + ol;
        uint32_t pk[4];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int c = cb * kHaloCB + kg * 8 + e;
            float v = 0.f;
            if (o < CO && c < CI)
                v = TR ? w[((size_t)c * CO + o) * 9 + (8 - tap)] : w[((size_t)o * CI + c) * 9 + tap];
            const uint32_t h = bf16_bits(v);
            pk[e >> 1] = (e & 1) ? (pk[e >> 1] | (h << 16)) : h;
        }
        unsigned char *dst = reinterpret_cast<unsigned char *>(wimg) + (size_t)blk * NT * kHaloCB * 2 + kmaj(ol, kg * 8);
        *reinterpret_cast<uint4 *>(dst) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
}

// Input rows i0 - 1 .. i0 + kHaloRows of channel block cb, pixels j0 - 1 ..
// j0 + 128, as BF16 (zeros outside the image and past CI): 16-byte row
// ((row * 4 + channel group) * kHaloQ + pixel). Consecutive threads take
// consecutive pixels, so each of the 8 loads of a row is coalesced.
__device__ __forceinline__ void stage_halo(unsigned char *hb, const float *__restrict__ xn, int cb, int CI, int H,
                                           int W, int i0, int j0)
{
    constexpr int items = (kHaloRows + 2) * (kHaloCB / 8) * kHaloQ;
    for (int it = threadIdx.x; it < items; it += kConvThreads) {
        const int q = it % kHaloQ, rest = it / kHaloQ;
        const int g = rest % (kHaloCB / 8), rr = rest / (kHaloCB / 8);
        const int row = i0 - 1 + rr, col = j0 - 1 + q, c0 = cb * kHaloCB + g * 8;
        const bool in = row >= 0 && row < H && col >= 0 && col < W;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e)
            v[e] = (in && c0 + e < CI) ? __ldg(xn + ((size_t)(c0 + e) * H + row) * W + col) : 0.f;
        uint32_t pk[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) pk[e] = bf16_bits(v[2 * e]) | (bf16_bits(v[2 * e + 1]) << 16);
        *reinterpret_cast<uint4 *>(hb + (size_t)it * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
}

__global__ void __launch_bounds__(kConvThreads) k_conv3x3_tc(const float *__restrict__ x,
                                                             const uint16_t *__restrict__ wimg,
                                                             const float *__restrict__ b, float *__restrict__ y,
                                                             int CI, int CO, int H, int W, int NT, unsigned *err)
{
    extern __shared__ __align__(1024) unsigned char nsm[];
    __shared__ __align__(8) uint64_t wfull[kWRing], wempty[kWRing], hdone[2], fin;
    __shared__ uint32_t tslot;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int ob = (CO + NT - 1) / NT;
    const int n = blockIdx.z / ob, obi = blockIdx.z % ob, o0 = obi * NT;
    const int i0 = blockIdx.y * kHaloRows, j0 = blockIdx.x * kRowsTc;
    const int ncb = (CI + kHaloCB - 1) / kHaloCB, nblk = ncb * 9;
    const int AS = acc_stride(NT);
    const uint32_t wbytes = (uint32_t)NT * kHaloCB * 2;
    unsigned char *halo[2] = {nsm, nsm + kHaloBytes};
    unsigned char *wring = nsm + 2 * kHaloBytes;
    const unsigned char *wsrc = reinterpret_cast<const unsigned char *>(wimg) + (size_t)obi * ncb * 9 * wbytes;
    if (t == 0) {
        for (int k = 0; k < kWRing; ++k) {
            nn_mbar_init(smem_addr(&wfull[k]), 1);
            nn_mbar_init(smem_addr(&wempty[k]), 1);
        }
        nn_mbar_init(smem_addr(&hdone[0]), 1);
        nn_mbar_init(smem_addr(&hdone[1]), 1);
        nn_mbar_init(smem_addr(&fin), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) nn_tmem_alloc(smem_addr(&tslot), (uint32_t)tmem_cols(kHaloRows * AS));
    nn_before_sync();
    __syncthreads();
    nn_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t id = nn_idesc(NT);
    int issued = 0;  // weight blocks whose copy thread 0 has issued
    if (t == 0)
        for (; issued < min(kWRing, nblk); ++issued) {
            nn_expect_tx(smem_addr(&wfull[issued]), wbytes);
            nn_bulk_g2s(smem_addr(wring + (size_t)issued * wbytes), wsrc + (size_t)issued * wbytes, wbytes,
                        smem_addr(&wfull[issued]));
        }
    const float *xn = x + (size_t)n * CI * H * W;
    stage_halo(halo[0], xn, 0, CI, H, W, i0, j0);
    nn_fence_async();
    bool ok = __syncthreads_and(1) != 0;
    for (int cb = 0; cb < ncb && ok; ++cb) {
        const unsigned char *hb = halo[cb & 1];
        if (t == 0) {
            for (int tap = 0; tap < 9 && ok; ++tap) {
                const int g = cb * 9 + tap, slot = g % kWRing;
                // the slot of block g - 2 takes block g - 2 + kWRing once that
                // block's MMAs are done (those of block g - 1 keep the pipe busy)
                if (g >= 2 && issued == g - 2 + kWRing && issued < nblk) {
                    const int ps = (g - 2) % kWRing;
                    ok = nn_wait(smem_addr(&wempty[ps]), (uint32_t)((g - 2) / kWRing) & 1u);
                    if (!ok) break;
                    nn_expect_tx(smem_addr(&wfull[ps]), wbytes);
                    nn_bulk_g2s(smem_addr(wring + (size_t)ps * wbytes), wsrc + (size_t)issued * wbytes, wbytes,
                                smem_addr(&wfull[ps]));
                    ++issued;
                }
                ok = nn_wait(smem_addr(&wfull[slot]), (uint32_t)(g / kWRing) & 1u);
                if (!ok) break;
                nn_after_sync();
                const int u = tap / 3, v = tap - 3 * (tap / 3);
                const uint32_t wb = smem_addr(wring + (size_t)slot * wbytes);
#pragma unroll
                for (int r = 0; r < kHaloRows; ++r)
#pragma unroll
                    for (int h = 0; h < kHaloCB / 16; ++h) {
                        const uint32_t a = smem_addr(hb) + (uint32_t)((((r + u) * (kHaloCB / 8) + 2 * h) * kHaloQ + v) * 16);
                        nn_mma(tmem + (uint32_t)(r * AS), halo_desc(a), nn_sdesc(wb + h * 256), id,
                               (cb > 0 || tap > 0 || h > 0) ? 1u : 0u);
                    }
                nn_commit(smem_addr(&wempty[slot]));
            }
            // completes once every MMA issued so far (all reading hb) is done
            nn_commit(smem_addr(&hdone[cb & 1]));
        }
        if (cb + 1 < ncb) {
            // the other buffer was read by the MMAs of block cb - 1
            if (cb >= 1) ok = ok && nn_wait(smem_addr(&hdone[(cb + 1) & 1]), (uint32_t)((cb - 1) >> 1) & 1u);
            if (ok) stage_halo(halo[(cb + 1) & 1], xn, cb + 1, CI, H, W, i0, j0);
            nn_fence_async();
        }
        ok = __syncthreads_and(ok) != 0;
    }
    // every MMA is done once the last block's commit has landed
    if (ok) ok = nn_wait(smem_addr(&hdone[(ncb - 1) & 1]), (uint32_t)((ncb - 1) >> 1) & 1u);
    ok = __syncthreads_and(ok) != 0;
    nn_after_sync();
    if (!ok) {
        if (t == 0) {
            // a wait gave up: the MMAs and the weight copies issued so far
            // land before the tensor memory and shared memory are released
            nn_commit(smem_addr(&fin));
            nn_wait(smem_addr(&fin), 0u);
            for (int g = max(0, issued - kWRing); g < issued; ++g)
                nn_wait(smem_addr(&wfull[g % kWRing]), (uint32_t)(g / kWRing) & 1u);
            atomicOr(err, 1u);
        }
    } else {
        // warp w: tensor-memory lanes (pixels) 32 (w % 4) .. + 31, output row w / 4
        const int q = warp & 3, r = warp >> 2;
        const int i = i0 + r, jp = j0 + 32 * q + lane;
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(r * AS);
        float *yn = y + (size_t)n * CO * H * W;
        for (int c0 = 0; c0 < NT; c0 += 32) {
            uint32_t rv[32];
            nn_ld32(tl + (uint32_t)c0, rv);
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const int o = o0 + c0 + e;
                if (c0 + e < NT && o < CO && i < H && jp < W)
                    yn[((size_t)o * H + i) * W + jp] = __uint_as_float(rv[e]) + (b ? __ldg(b + o) : 0.f);
            }
        }
    }
    nn_before_sync();
    __syncthreads();
    nn_after_sync();
    if (warp == 0) nn_tmem_free(tmem, (uint32_t)tmem_cols(kHaloRows * AS));
}

// ---------------------------------------------------------------------------
// Weight and bias gradient. CTA: all output channels (rows, CO <= 128),
// columns kc0 .. kc0 + NC - 1 of the CI * 9 + 1 (input channel, tap) columns
// (the last is the bias: a column of ones), pixels p_lo .. p_hi of the
// flattened B x H x W pixels (K). Writes its partial sums to
// part[split][o][column].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_conv3x3_dw_tc(const float *__restrict__ x, const float *__restrict__ dy,
                                                        float *__restrict__ part, int CI, int CO, int H, int W,
                                                        int64_t P, int64_t per_split, int NC, unsigned *err)
{
    extern __shared__ __align__(1024) unsigned char nsm[];
    __shared__ __align__(8) uint64_t done[2], fin;
    __shared__ uint32_t tslot;
    __shared__ int pn[kKB], pi[kKB], pj[kKB];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int ncol = CI * 9 + 1, kc0 = blockIdx.x * NC, split = blockIdx.y;
    const int64_t p_lo = (int64_t)split * per_split, p_hi = min(P, p_lo + per_split);
    const int nblk = p_hi > p_lo ? (int)((p_hi - p_lo + kKB - 1) / kKB) : 0;
    const int bbytes = NC * kKB * 2;
    unsigned char *stage[2] = {nsm, nsm + kABytes + bbytes};
    if (t == 0) {
        nn_mbar_init(smem_addr(&done[0]), 1);
        nn_mbar_init(smem_addr(&done[1]), 1);
        nn_mbar_init(smem_addr(&fin), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) nn_tmem_alloc(smem_addr(&tslot), (uint32_t)tmem_cols(NC));
    nn_before_sync();
    __syncthreads();
    nn_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t id = nn_idesc(NC);
    const int64_t HW = (int64_t)H * W;
    bool ok = true;
    for (int kb = 0; kb < nblk; ++kb) {
        const int sg = kb & 1;
        if (kb >= 2) ok = ok && nn_wait(smem_addr(&done[sg]), (uint32_t)((kb - 2) >> 1) & 1u);
        // the block's 32 pixels (image, row, column; -1: past the range)
        if (t < kKB) {
            const int64_t p = p_lo + (int64_t)kb * kKB + t;
            if (p < p_hi) {
                const int64_t nimg = p / HW, r = p - nimg * HW;
                pn[t] = (int)nimg;
                pi[t] = (int)(r / W);
                pj[t] = (int)(r - (r / W) * W);
            } else {
                pn[t] = -1;
            }
        }
        __syncthreads();
        unsigned char *sa = stage[sg], *sb = sa + kABytes;
        // A: output channel t over the 32 pixels, 8 per 16-byte row
#pragma unroll
        for (int g = 0; g < kKB / 8; ++g) {
            uint32_t pk[4];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int kk = 8 * g + e;
                float v = 0.f;
                if (t < CO && pn[kk] >= 0)
                    v = __ldg(dy + (((size_t)pn[kk] * CO + t) * H + pi[kk]) * W + pj[kk]);
                const uint32_t h = bf16_bits(v);
                pk[e >> 1] = (e & 1) ? (pk[e >> 1] | (h << 16)) : h;
            }
            *reinterpret_cast<uint4 *>(sa + kmaj(t, 8 * g)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
        // B: columns kc0 + t and kc0 + t + 128 over the 32 pixels
        for (int row = t; row < NC; row += 128) {
            const int col = kc0 + row;
            const int c = col / 9, uv = col - 9 * c, u = uv / 3, vv = uv - 3 * u;
#pragma unroll
            for (int g = 0; g < kKB / 8; ++g) {
                uint32_t pk[4];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int kk = 8 * g + e;
                    float v = 0.f;
                    if (pn[kk] >= 0 && col < ncol) {
                        if (col == ncol - 1) {
                            v = 1.f;  // the bias column
                        } else {
                            const int ii = pi[kk] + u - 1, jj = pj[kk] + vv - 1;
                            if (ii >= 0 && ii < H && jj >= 0 && jj < W)
                                v = __ldg(x + (((size_t)pn[kk] * CI + c) * H + ii) * W + jj);
                        }
                    }
                    const uint32_t h = bf16_bits(v);
                    pk[e >> 1] = (e & 1) ? (pk[e >> 1] | (h << 16)) : h;
                }
                *reinterpret_cast<uint4 *>(sb + kmaj(row, 8 * g)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
        }
        nn_fence_async();
        nn_before_sync();
        ok = __syncthreads_and(ok) != 0;  // every thread's stage was free
        nn_after_sync();
        if (t == 0 && ok) {
#pragma unroll
            for (int kk = 0; kk < kKB; kk += 16)
                nn_mma(tmem, nn_sdesc(smem_addr(sa) + kk * 16), nn_sdesc(smem_addr(sb) + kk * 16), id,
                       (kb > 0 || kk > 0) ? 1u : 0u);
            nn_commit(smem_addr(&done[sg]));
        }
    }
    if (nblk > 0) {
        const int last = nblk - 1;
        ok = ok && nn_wait(smem_addr(&done[last & 1]), (uint32_t)(last >> 1) & 1u);
    }
    ok = __syncthreads_and(ok) != 0;
    nn_after_sync();
    if (!ok) {
        if (t == 0) {
            nn_commit(smem_addr(&fin));
            nn_wait(smem_addr(&fin), 0u);
            atomicOr(err, 1u);
        }
    } else {
        // warp w holds output channels 32 w .. 32 w + 31
        const int o = 32 * warp + lane;
        const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
        for (int c0 = 0; c0 < NC; c0 += 32) {
            uint32_t r[32];
            if (nblk > 0) nn_ld32(tl + (uint32_t)c0, r);
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const int col = kc0 + c0 + e;
                if (o < CO && c0 + e < NC && col < ncol)
                    part[((size_t)split * CO + o) * ncol + col] = nblk > 0 ? __uint_as_float(r[e]) : 0.f;
            }
        }
    }
    nn_before_sync();
    __syncthreads();
    nn_after_sync();
    if (warp == 0) nn_tmem_free(tmem, (uint32_t)tmem_cols(NC));
}

// dw[o][c][u][v] and db[o] = the splits' partial sums, added in split order.
__global__ void k_conv3x3_dw_tc_sum(const float *__restrict__ part, float *__restrict__ dw, float *__restrict__ db,
                                    int CI, int CO, int S)
{
    const int ncol = CI * 9 + 1;
    const int64_t n = (int64_t)CO * ncol;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int s = 0; s < S; ++s) acc += part[(size_t)s * n + e];
        const int o = (int)(e / ncol), col = (int)(e - (int64_t)o * ncol);
        if (col < ncol - 1) dw[(size_t)o * (ncol - 1) + col] = acc;
        else db[o] = acc;
    }
}

__device__ unsigned g_nn_tc_err;  // a tensor-core layer's wait gave up (dg_nn_tc_check)

namespace {

int nt_of(int co) { return std::min(128, (co + 15) / 16 * 16); }
int nc_of(int ci) { return std::min(256, (ci * 9 + 1 + 15) / 16 * 16); }

int64_t dw_splits(int B, int Ci, int Co, int H, int W)
{
    const int64_t P = (int64_t)B * H * W;
    const int64_t tiles = (Ci * 9 + 1 + nc_of(Ci) - 1) / nc_of(Ci);
    int64_t S = (152 * 4 + tiles - 1) / tiles;          // about four CTAs per SM
    S = std::min<int64_t>(S, std::max<int64_t>(1, P / 1024));
    return std::max<int64_t>(1, std::min<int64_t>(S, 4096));
}

bool tc_shape_ok(int B, int Ci, int Co, int H, int W)
{
    return B > 0 && Ci > 0 && Co > 0 && H > 0 && W > 0 && Ci <= 4096 && Co <= 4096 && H <= 65535 &&
           (int64_t)B * ((Co + 127) / 128) <= 65535 && (int64_t)B * std::max(Ci, Co) * H * W <= ((int64_t)1 << 40);
}

unsigned *err_word()
{
    void *p = nullptr;
    return cudaGetSymbolAddress(&p, g_nn_tc_err) == cudaSuccess ? (unsigned *)p : nullptr;
}

cudaError_t launch_conv_tc(bool tr, const float *x, const float *w, const float *b, float *y, int B, int CI, int CO,
                           int H, int W, uint16_t *wimg, cudaStream_t s)
{
    unsigned *err = err_word();
    if (!err) return cudaErrorInvalidSymbol;
    const int NT = nt_of(CO);
    const int64_t items = wimg_elems(CI, CO, NT) / 8;
    const unsigned gw = (unsigned)std::min<int64_t>((items + 255) / 256, 152 * 8);
    if (tr) k_conv_tc_wimg<true><<<gw, 256, 0, s>>>(w, wimg, CI, CO, NT);
    else k_conv_tc_wimg<false><<<gw, 256, 0, s>>>(w, wimg, CI, CO, NT);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int smem = conv_tc_smem(NT);
    if ((e = cudaFuncSetAttribute(k_conv3x3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
        return e;
    const dim3 grid((W + kRowsTc - 1) / kRowsTc, (H + kHaloRows - 1) / kHaloRows, B * ((CO + NT - 1) / NT));
    k_conv3x3_tc<<<grid, kConvThreads, smem, s>>>(x, wimg, b, y, CI, CO, H, W, NT, err);
    return cudaGetLastError();
}

// floats of scratch: the forward's weight blocks, or the backward's (data
// gradient weight blocks, then the weight gradient's partial sums)
int64_t fwd_scratch(int Ci, int Co) { return (wimg_elems(Ci, Co, nt_of(Co)) + 7) / 8 * 4; }
int64_t bwd_wimg_floats(int Ci, int Co) { return (wimg_elems(Co, Ci, nt_of(Ci)) + 7) / 8 * 4; }

}  // namespace

int64_t nn_conv_tc_scratch(int B, int Ci, int Co, int H, int W)
{
    return std::max(fwd_scratch(Ci, Co), bwd_wimg_floats(Ci, Co) + dw_splits(B, Ci, Co, H, W) * (int64_t)Co * (Ci * 9 + 1));
}

}  // namespace dg

extern "C" {

dg_status dg_nn_conv3x3_forward_tc(const float *x, const float *w, const float *b, float *y, int32_t B, int32_t Ci,
                                   int32_t Co, int32_t H, int32_t W, float *scratch, void *stream)
{
    if (!x || !w || !b || !y || !scratch) return dg::nn_fail(DG_EINVAL, "dg_nn_conv3x3_forward_tc: null pointer");
    if (!dg::tc_shape_ok(B, Ci, Co, H, W))
        return dg::nn_fail(DG_EINVAL, "dg_nn_conv3x3_forward_tc: bad shape B=%d Ci=%d Co=%d H=%d W=%d", B, Ci, Co, H, W);
    if ((reinterpret_cast<uintptr_t>(scratch) & 15) != 0)
        return dg::nn_fail(DG_EINVAL, "dg_nn_conv3x3_forward_tc: scratch must be 16-byte aligned");
    return dg::nn_done(dg::launch_conv_tc(false, x, w, b, y, B, Ci, Co, H, W, reinterpret_cast<uint16_t *>(scratch),
                                          (cudaStream_t)stream),
                       "dg_nn_conv3x3_forward_tc");
}

int64_t dg_nn_conv3x3_tc_scratch(int32_t B, int32_t Ci, int32_t Co, int32_t H, int32_t W)
{
    if (!dg::tc_shape_ok(B, Ci, Co, H, W)) return -1;
    if (Co > 128) return dg::fwd_scratch(Ci, Co);  // the backward refuses this shape
    return dg::nn_conv_tc_scratch(B, Ci, Co, H, W);
}

dg_status dg_nn_conv3x3_backward_tc(const float *x, const float *w, const float *dy, float *dx, float *dw, float *db,
                                    int32_t B, int32_t Ci, int32_t Co, int32_t H, int32_t W, float *scratch,
                                    void *stream)
{
    if (!x || !w || !dy || !dw || !db || !scratch)
        return dg::nn_fail(DG_EINVAL, "dg_nn_conv3x3_backward_tc: null pointer");
    if (!dg::tc_shape_ok(B, Ci, Co, H, W))
        return dg::nn_fail(DG_EINVAL, "dg_nn_conv3x3_backward_tc: bad shape B=%d Ci=%d Co=%d H=%d W=%d", B, Ci, Co, H, W);
    if (Co > 128)
        return dg::nn_fail(DG_EUNSUPPORTED, "dg_nn_conv3x3_backward_tc: at most 128 output channels (Co=%d)", Co);
    if ((reinterpret_cast<uintptr_t>(scratch) & 15) != 0)
        return dg::nn_fail(DG_EINVAL, "dg_nn_conv3x3_backward_tc: scratch must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (dx) e = dg::launch_conv_tc(true, dy, w, nullptr, dx, B, Co, Ci, H, W, reinterpret_cast<uint16_t *>(scratch), s);
    float *part = scratch + dg::bwd_wimg_floats(Ci, Co);
    if (e != cudaSuccess) return dg::nn_done(e, "dg_nn_conv3x3_backward_tc");
    unsigned *err = dg::err_word();
    if (!err) return dg::nn_done(cudaErrorInvalidSymbol, "dg_nn_conv3x3_backward_tc");
    const int NC = dg::nc_of(Ci);
    const int64_t S = dg::dw_splits(B, Ci, Co, H, W);
    const int64_t P = (int64_t)B * H * W;
    const int64_t per = (P + S - 1) / S;
    const int smem = 2 * (dg::kABytes + NC * dg::kKB * 2);
    if ((e = cudaFuncSetAttribute(dg::k_conv3x3_dw_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
        return dg::nn_done(e, "dg_nn_conv3x3_backward_tc");
    const dim3 grid((unsigned)((Ci * 9 + 1 + NC - 1) / NC), (unsigned)S);
    dg::k_conv3x3_dw_tc<<<grid, 128, smem, s>>>(x, dy, part, Ci, Co, H, W, P, per, NC, err);
    if ((e = cudaGetLastError()) != cudaSuccess) return dg::nn_done(e, "dg_nn_conv3x3_backward_tc");
    const int64_t n = (int64_t)Co * (Ci * 9 + 1);
    dg::k_conv3x3_dw_tc_sum<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, s>>>(part, dw, db, Ci,
                                                                                                  Co, (int)S);
    return dg::nn_done(cudaGetLastError(), "dg_nn_conv3x3_backward_tc");
}

dg_status dg_nn_tc_check(void *stream)
{
    unsigned *err = dg::err_word();
    if (!err) return dg::nn_fail(DG_ECUDA, "dg_nn_tc_check: the error word has no device address");
    unsigned h = 0;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&h, err, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return dg::nn_done(e, "dg_nn_tc_check");
    if (h) {
        cudaMemsetAsync(err, 0, sizeof h, s);
        cudaStreamSynchronize(s);
        return dg::nn_fail(DG_ETIMEOUT, "a tensor-core layer's wait ran out; its outputs are not valid");
    }
    return DG_OK;
}

}  // extern "C"
