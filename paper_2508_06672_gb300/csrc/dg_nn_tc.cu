// dg_nn_tc.cu -- the proposal network's 3 x 3 convolutions on the tensor
// cores (tcgen05, sm_103a): BF16 activations and weights, FP32 accumulation.
//
// Both are implicit GEMMs with the accumulator in tensor memory and the
// operands staged in shared memory (no swizzle, K-major canonical layout:
// 8-row x 16-byte core matrices, 128 B apart along K and 512 B apart along
// the rows, in blocks of 32 K elements):
//
//   forward / data gradient: rows = 128 consecutive pixels of one image
//     row, columns = output channels, K = (input channel, tap) pairs:
//       y[n,o,i,j] = b[o] + sum_{c,u,v} w[o,c,u,v] x[n,c,i+u-1,j+v-1]
//     The data gradient is the same product with dy as the input, the
//     weights transposed (input and output channels swapped) and the taps
//     flipped:
//       dx[n,c,i,j] = sum_{o,u,v} w[o,c,u,v] dy[n,o,i-u+1,j-v+1]
//   weight gradient: rows = output channels, columns = (input channel, tap)
//     pairs plus one column of ones (the bias gradient), K = pixels:
//       dw[o,c,u,v] = sum_{n,i,j} dy[n,o,i,j] x[n,c,i+u-1,j+v-1]
//       db[o]       = sum_{n,i,j} dy[n,o,i,j]
//     split over pixel ranges; the partial sums are added in a fixed order.
//
// Every CTA: 128 threads gather a 32-element K block of both operands
// (rounded to BF16) into one of two shared-memory stages, one thread issues
// the MMAs of the block and commits them to that stage's mbarrier, and the
// next block is gathered into the other stage meanwhile. The gathers are
// plain loads from L2; the FP32 kernels in dg_nn.cu stay as the reference.
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
// Forward (TR = false) and data gradient (TR = true). CTA: pixels j0 .. j0 +
// 127 of row i of image n, output channels o0 .. o0 + NT - 1 (NT a multiple
// of 16, <= 128, from blockIdx.z). x: [B][CI][H][W]; y: [B][CO][H][W]; w:
// [CO][CI][3][3] (forward) or the forward convolution's [CI][CO][3][3]
// (data gradient, read transposed with flipped taps); b may be NULL.
// ---------------------------------------------------------------------------
template <bool TR>
__global__ void __launch_bounds__(128) k_conv3x3_tc(const float *__restrict__ x, const float *__restrict__ w,
                                                     const float *__restrict__ b, float *__restrict__ y, int CI,
                                                     int CO, int H, int W, int NT, unsigned *err)
{
    extern __shared__ __align__(1024) unsigned char nsm[];
    __shared__ __align__(8) uint64_t done[2], fin;
    __shared__ uint32_t tslot;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int ob = (CO + NT - 1) / NT;
    const int n = blockIdx.z / ob, o0 = (blockIdx.z % ob) * NT;
    const int i = blockIdx.y, j0 = blockIdx.x * kRowsTc;
    const int K = CI * 9, nblk = (K + kKB - 1) / kKB;
    const int bbytes = NT * kKB * 2;
    unsigned char *stage[2] = {nsm, nsm + kABytes + bbytes};
    if (t == 0) {
        nn_mbar_init(smem_addr(&done[0]), 1);
        nn_mbar_init(smem_addr(&done[1]), 1);
        nn_mbar_init(smem_addr(&fin), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) nn_tmem_alloc(smem_addr(&tslot), (uint32_t)tmem_cols(NT));
    nn_before_sync();
    __syncthreads();
    nn_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t id = nn_idesc(NT);
    const float *xn = x + (size_t)n * CI * H * W;
    const int j = j0 + t;  // this thread's pixel (A row)
    bool ok = true;
    for (int kb = 0; kb < nblk; ++kb) {
        const int sg = kb & 1;
        // the stage's previous MMAs (block kb - 2) are done before it is rewritten
        if (kb >= 2) ok = ok && nn_wait(smem_addr(&done[sg]), (uint32_t)((kb - 2) >> 1) & 1u);
        unsigned char *sa = stage[sg], *sb = sa + kABytes;
        // A: this pixel's 32 (channel, tap) values, 8 at a time into one
        // 16-byte core-matrix row; (channel, tap) stepped from the block's start
        {
            int k = kb * kKB, c = k / 9, uv = k - 9 * c;
#pragma unroll
            for (int g = 0; g < kKB / 8; ++g) {
                uint32_t pk[4];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    float v = 0.f;
                    if (k < K && j < W) {
                        const int u = uv / 3, vv = uv - 3 * u;
                        const int ii = i + u - 1, jj = j + vv - 1;
                        if (ii >= 0 && ii < H && jj >= 0 && jj < W) v = __ldg(xn + ((size_t)c * H + ii) * W + jj);
                    }
                    const uint32_t h = bf16_bits(v);
                    pk[e >> 1] = (e & 1) ? (pk[e >> 1] | (h << 16)) : h;
                    ++k;
                    if (++uv == 9) {
                        uv = 0;
                        ++c;
                    }
                }
                *reinterpret_cast<uint4 *>(sa + kmaj(t, 8 * g)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
        }
        // B: output channel o0 + t's 32 weights, likewise
        if (t < NT) {
            const int o = o0 + t;
            int k = kb * kKB, ci = k / 9, uv = k - 9 * ci;
#pragma unroll
            for (int g = 0; g < kKB / 8; ++g) {
                uint32_t pk[4];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    float v = 0.f;
                    if (k < K && o < CO)
                        v = TR ? __ldg(w + ((size_t)ci * CO + o) * 9 + (8 - uv))  // w[ci][o][2-u][2-v]
                               : __ldg(w + (size_t)o * K + k);
                    const uint32_t h = bf16_bits(v);
                    pk[e >> 1] = (e & 1) ? (pk[e >> 1] | (h << 16)) : h;
                    ++k;
                    if (++uv == 9) {
                        uv = 0;
                        ++ci;
                    }
                }
                *reinterpret_cast<uint4 *>(sb + kmaj(t, 8 * g)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
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
    // every MMA is done once the last block's commit has landed
    const int last = nblk - 1;
    ok = ok && nn_wait(smem_addr(&done[last & 1]), (uint32_t)(last >> 1) & 1u);
    ok = __syncthreads_and(ok) != 0;
    nn_after_sync();
    if (!ok) {
        if (t == 0) {
            // a wait gave up: the MMAs issued so far land before the tensor
            // memory is freed
            nn_commit(smem_addr(&fin));
            nn_wait(smem_addr(&fin), 0u);
            atomicOr(err, 1u);
        }
    } else {
        // warp w holds pixels 32 w .. 32 w + 31 (its tensor-memory lanes)
        const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
        const int jp = j0 + 32 * warp + lane;
        float *yn = y + (size_t)n * CO * H * W;
        for (int c0 = 0; c0 < NT; c0 += 32) {
            uint32_t r[32];
            nn_ld32(tl + (uint32_t)c0, r);
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const int o = o0 + c0 + e;
                if (c0 + e < NT && o < CO && jp < W)
                    yn[((size_t)o * H + i) * W + jp] = __uint_as_float(r[e]) + (b ? __ldg(b + o) : 0.f);
            }
        }
    }
    nn_before_sync();
    __syncthreads();
    nn_after_sync();
    if (warp == 0) nn_tmem_free(tmem, (uint32_t)tmem_cols(NT));
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
                           int H, int W, cudaStream_t s)
{
    unsigned *err = err_word();
    if (!err) return cudaErrorInvalidSymbol;
    const int NT = nt_of(CO);
    const int smem = 2 * (kABytes + NT * kKB * 2);
    const dim3 grid((W + kRowsTc - 1) / kRowsTc, H, B * ((CO + NT - 1) / NT));
    cudaError_t e;
    if (tr) {
        if ((e = cudaFuncSetAttribute(k_conv3x3_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
            return e;
        k_conv3x3_tc<true><<<grid, 128, smem, s>>>(x, w, b, y, CI, CO, H, W, NT, err);
    } else {
        if ((e = cudaFuncSetAttribute(k_conv3x3_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
            return e;
        k_conv3x3_tc<false><<<grid, 128, smem, s>>>(x, w, b, y, CI, CO, H, W, NT, err);
    }
    return cudaGetLastError();
}

}  // namespace

int64_t nn_conv_tc_scratch(int B, int Ci, int Co, int H, int W)
{
    return dw_splits(B, Ci, Co, H, W) * (int64_t)Co * (Ci * 9 + 1);
}

}  // namespace dg

extern "C" {

dg_status dg_nn_conv3x3_forward_tc(const float *x, const float *w, const float *b, float *y, int32_t B, int32_t Ci,
                                   int32_t Co, int32_t H, int32_t W, void *stream)
{
    if (!x || !w || !b || !y) return dg::nn_fail(DG_EINVAL, "dg_nn_conv3x3_forward_tc: null pointer");
    if (!dg::tc_shape_ok(B, Ci, Co, H, W))
        return dg::nn_fail(DG_EINVAL, "dg_nn_conv3x3_forward_tc: bad shape B=%d Ci=%d Co=%d H=%d W=%d", B, Ci, Co, H, W);
    return dg::nn_done(dg::launch_conv_tc(false, x, w, b, y, B, Ci, Co, H, W, (cudaStream_t)stream),
                       "dg_nn_conv3x3_forward_tc");
}

int64_t dg_nn_conv3x3_tc_scratch(int32_t B, int32_t Ci, int32_t Co, int32_t H, int32_t W)
{
    if (!dg::tc_shape_ok(B, Ci, Co, H, W) || Co > 128) return -1;
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
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (dx) e = dg::launch_conv_tc(true, dy, w, nullptr, dx, B, Co, Ci, H, W, s);
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
    dg::k_conv3x3_dw_tc<<<grid, 128, smem, s>>>(x, dy, scratch, Ci, Co, H, W, P, per, NC, err);
    if ((e = cudaGetLastError()) != cudaSuccess) return dg::nn_done(e, "dg_nn_conv3x3_backward_tc");
    const int64_t n = (int64_t)Co * (Ci * 9 + 1);
    dg::k_conv3x3_dw_tc_sum<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, s>>>(scratch, dw, db, Ci,
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
