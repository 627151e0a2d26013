// dg_nn.cu -- the layers of the learned proposal network, forward and
// backward, FP32 (NCHW tensors in device memory).
//
//   conv3x3   3 x 3 cross-correlation, zero padding 1, stride 1, bias:
//             y[n,o,i,j] = b[o] + sum_c sum_{u,v} w[o,c,u,v] x[n,c,i+u-1,j+v-1]
//   backward  dx[n,c,i,j] = sum_o sum_{u,v} w[o,c,u,v] dy[n,o,i-u+1,j-v+1]
//             dw[o,c,u,v] = sum_{n,i,j} dy[n,o,i,j] x[n,c,i+u-1,j+v-1]
//             db[o]       = sum_{n,i,j} dy[n,o,i,j]
//   relu, its backward, the weighted binary cross-entropy on logits (loss and
//   gradient), and one Adam step.
//
// The convolutions are direct, FP32: each CTA stages a 16 x 32 pixel tile
// of one input channel (with its halo) and the matching 3 x 3 x 16 weights in
// shared memory and accumulates 16 output channels over all input channels;
// the data gradient is the same kernel on the flipped, transposed weights.
// The weight and bias gradients are summed per (8 output channels, input
// channel, pixel split), then over the splits in a fixed order, so every
// result is deterministic.
#include <algorithm>
#include <cstdarg>
#include <cstdio>

#include "dg_internal.cuh"

namespace dg {

namespace {
// Convolution tiles: a CTA of 128 threads computes a 16 x 32 pixel tile of
// 16 output channels; thread (ty, tx) owns 4 neighbouring pixels of row ty
// for all 16 channels (64 accumulators). Per input channel the 18 x 34 input
// window (with its halo) and the 9 x 16 weights sit in shared memory; per
// kernel row a thread reads 6 inputs and, per tap, 16 weights (4 float4
// broadcasts) for 64 FMAs.
constexpr int kTH = 16, kTW = 32, kOC = 16, kPX = 4;
constexpr int kXR = kTH + 2, kXC = kTW + 2, kXS = kTW + 4;  // window rows, columns, row stride

// y = conv(x) (+ b), or, with TR, the data gradient of a convolution: then x
// is dy (CI = that convolution's output channels), y is dx (CO = its input
// channels) and w keeps that convolution's [CI][CO][3][3] layout, read with
// the taps flipped.
template <bool TR>
__global__ void __launch_bounds__(128) k_conv3x3_tiled(const float *__restrict__ x, const float *__restrict__ w,
                                                        const float *__restrict__ b, float *__restrict__ y, int CI,
                                                        int CO, int H, int W)
{
    // per-thread shares of the window (kXR x kXC) and of the weights (9 x kOC)
    constexpr int kXPer = (kXR * kXC + 127) / 128, kWPer = (9 * kOC + 127) / 128;
    __shared__ __align__(16) float xs[kXR][kXS];
    __shared__ __align__(16) float ws[9][kOC];
    const int ocb = (CO + kOC - 1) / kOC;
    const int n = blockIdx.z / ocb, oc0 = (blockIdx.z % ocb) * kOC;
    const int i0 = blockIdx.y * kTH, j0 = blockIdx.x * kTW;
    const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
    // the window elements and weights this thread stages, resolved once:
    // source offset within a channel plane (or -1: zero padding) and slot
    int xoff[kXPer], xslot[kXPer], woff[kWPer], wslot[kWPer];
#pragma unroll
    for (int e = 0; e < kXPer; ++e) {
        const int idx = threadIdx.x + 128 * e;
        const int r = idx / kXC, cc = idx % kXC;
        const int gi = i0 + r - 1, gj = j0 + cc - 1;
        xslot[e] = idx < kXR * kXC ? r * kXS + cc : -1;
        xoff[e] = (idx < kXR * kXC && gi >= 0 && gi < H && gj >= 0 && gj < W) ? gi * W + gj : -1;
    }
#pragma unroll
    for (int e = 0; e < kWPer; ++e) {
        const int idx = threadIdx.x + 128 * e;
        const int t = idx / kOC, o = idx % kOC, oc = oc0 + o;
        wslot[e] = idx < 9 * kOC ? t * kOC + o : -1;
        woff[e] = (idx < 9 * kOC && oc < CO) ? (TR ? oc * 9 + (8 - t) : oc * CI * 9 + t) : -1;
    }
    const size_t plane = (size_t)H * W;
    const float *xn = x + (size_t)n * CI * plane;
    // weight of (oc, ic, tap): w[(oc CI + ic) 9 + tap]; transposed: w[(ic CO + oc) 9 + 8 - tap]
    const size_t wstep = TR ? (size_t)CO * 9 : 9;
    float px[kXPer], pw[kWPer];
#pragma unroll
    for (int e = 0; e < kXPer; ++e) px[e] = xoff[e] >= 0 ? __ldg(xn + xoff[e]) : 0.f;
#pragma unroll
    for (int e = 0; e < kWPer; ++e) pw[e] = woff[e] >= 0 ? __ldg(w + woff[e]) : 0.f;
    float acc[kOC][kPX];
#pragma unroll
    for (int o = 0; o < kOC; ++o)
#pragma unroll
        for (int p = 0; p < kPX; ++p) acc[o][p] = 0.f;
    for (int ic = 0; ic < CI; ++ic) {
        __syncthreads();
#pragma unroll
        for (int e = 0; e < kXPer; ++e)
            if (xslot[e] >= 0) (&xs[0][0])[xslot[e]] = px[e];
#pragma unroll
        for (int e = 0; e < kWPer; ++e)
            if (wslot[e] >= 0) (&ws[0][0])[wslot[e]] = pw[e];
        __syncthreads();
        if (ic + 1 < CI) {  // the next channel's loads, in flight during this channel's FMAs
            const float *xc = xn + (size_t)(ic + 1) * plane;
            const float *wc = w + (size_t)(ic + 1) * wstep;
#pragma unroll
            for (int e = 0; e < kXPer; ++e) px[e] = xoff[e] >= 0 ? __ldg(xc + xoff[e]) : 0.f;
#pragma unroll
            for (int e = 0; e < kWPer; ++e) pw[e] = woff[e] >= 0 ? __ldg(wc + woff[e]) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const float4 xa = *reinterpret_cast<const float4 *>(&xs[ty + u][4 * tx]);
            const float2 xb = *reinterpret_cast<const float2 *>(&xs[ty + u][4 * tx + 4]);
            const float xr[6] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y};
#pragma unroll
            for (int v = 0; v < 3; ++v) {
#pragma unroll
                for (int o4 = 0; o4 < kOC / 4; ++o4) {
                    const float4 wv = *reinterpret_cast<const float4 *>(&ws[3 * u + v][4 * o4]);
                    const float wo[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q)
#pragma unroll
                        for (int p = 0; p < kPX; ++p) acc[4 * o4 + q][p] = fmaf(wo[q], xr[p + v], acc[4 * o4 + q][p]);
                }
            }
        }
    }
    const int i = i0 + ty;
    if (i >= H) return;
#pragma unroll
    for (int o = 0; o < kOC; ++o) {
        const int oc = oc0 + o;
        if (oc >= CO) break;
        const float bias = b ? __ldg(b + oc) : 0.f;
        float *yr = y + (((size_t)n * CO + oc) * H + i) * W;
#pragma unroll
        for (int p = 0; p < kPX; ++p) {
            const int j = j0 + 4 * tx + p;
            if (j < W) yr[j] = acc[o][p] + bias;
        }
    }
}

// Weight and bias gradients, first pass: CTA (o-block of 8, input channel c,
// pixel split s) sums dy[n,o,p] x[n,c,p + tap] over its share of the B*H*W
// pixels, 9 taps x 8 output channels per thread, then a fixed-order
// reduction over the CTA; partial[s][o][c][tap] (and, for c = 0,
// partial_b[s][o]).
constexpr int kDwO = 8;

__global__ void __launch_bounds__(256) k_conv3x3_dw(const float *__restrict__ x, const float *__restrict__ dy,
                                                     float *__restrict__ part, float *__restrict__ part_b, int B,
                                                     int Ci, int Co, int H, int W, int S)
{
    __shared__ float red[8][kDwO * 10];
    const int ob = blockIdx.x, c = blockIdx.y, s = blockIdx.z;
    const int o0 = ob * kDwO;
    const int64_t HW = (int64_t)H * W, P = (int64_t)B * HW;
    const int64_t p0 = P * s / S, p1 = P * (s + 1) / S;
    float acc[kDwO][10];  // 9 taps + the bias term
#pragma unroll
    for (int o = 0; o < kDwO; ++o)
#pragma unroll
        for (int t = 0; t < 10; ++t) acc[o][t] = 0.f;
    for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const int64_t n = p / HW, q = p % HW;
        const int i = (int)(q / W), j = (int)(q % W);
        const float *xc = x + ((size_t)n * Ci + c) * HW;
        float xv[9];
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                const int ii = i + u - 1, jj = j + v - 1;
                xv[3 * u + v] = (ii >= 0 && ii < H && jj >= 0 && jj < W) ? __ldg(xc + (size_t)ii * W + jj) : 0.f;
            }
#pragma unroll
        for (int o = 0; o < kDwO; ++o) {
            if (o0 + o >= Co) break;
            const float g = __ldg(dy + ((size_t)n * Co + o0 + o) * HW + q);
#pragma unroll
            for (int t = 0; t < 9; ++t) acc[o][t] = fmaf(g, xv[t], acc[o][t]);
            acc[o][9] += g;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 0; o < kDwO; ++o)
#pragma unroll
        for (int t = 0; t < 10; ++t) {
            float v = acc[o][t];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
            if (lane == 0) red[warp][o * 10 + t] = v;
        }
    __syncthreads();
    for (int e = threadIdx.x; e < kDwO * 10; e += blockDim.x) {
        const int o = e / 10, t = e % 10;
        if (o0 + o >= Co) continue;
        float v = 0.f;
        for (int q = 0; q < 8; ++q) v += red[q][e];
        if (t < 9) part[(((size_t)s * Co + o0 + o) * Ci + c) * 9 + t] = v;
        else if (c == 0) part_b[(size_t)s * Co + o0 + o] = v;
    }
}

// Second pass: dw = sum over splits in order; db likewise.
__global__ void k_conv3x3_dw_sum(const float *__restrict__ part, const float *__restrict__ part_b,
                                 float *__restrict__ dw, float *__restrict__ db, int Co, int Ci, int S)
{
    const int64_t nw = (int64_t)Co * Ci * 9;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nw + Co; e += (int64_t)gridDim.x * blockDim.x) {
        float v = 0.f;
        if (e < nw) {
            for (int s = 0; s < S; ++s) v += part[(size_t)s * nw + e];
            dw[e] = v;
        } else {
            const int64_t o = e - nw;
            for (int s = 0; s < S; ++s) v += part_b[(size_t)s * Co + o];
            db[o] = v;
        }
    }
}

// Fixed-order block sum of V values per thread (256 threads).
template <int V>
__device__ __forceinline__ void block_sum(float (&v)[V], float (&out)[V])
{
    __shared__ float sm[8][V];
#pragma unroll
    for (int k = 0; k < V; ++k)
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], d);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < V; ++k) sm[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < V; ++k) {
            float s = 0.f;
            for (int q = 0; q < 8; ++q) s += sm[q][k];
            out[k] = s;
        }
}

__global__ void k_relu_fwd(const float *__restrict__ z, float *__restrict__ h, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        h[t] = fmaxf(z[t], 0.f);
}

__global__ void k_relu_bwd(const float *__restrict__ z, const float *__restrict__ dh, float *__restrict__ dz, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        dz[t] = z[t] > 0.f ? dh[t] : 0.f;
}

// Weighted BCE on logits: per element the loss term and its gradient (both
// divided by n); loss partials per CTA, summed in a fixed order by one CTA.
__global__ void __launch_bounds__(256) k_bce(const float *__restrict__ z, const float *__restrict__ t, float pw,
                                              int64_t n, float *__restrict__ grad, float *__restrict__ part)
{
    float acc[1] = {0.f};
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float zz = z[k], tt = t[k];
        // log sigmoid(z) = -softplus(-z), log(1 - sigmoid(z)) = -softplus(z)
        const float sp_pos = fmaxf(zz, 0.f) + log1pf(expf(-fabsf(zz)));  // softplus(z)
        const float sp_neg = sp_pos - zz;                                  // softplus(-z)
        acc[0] += pw * tt * sp_neg + (1.f - tt) * sp_pos;
        // s(z) - 1 = -s(-z), formed directly so that it keeps its digits at large z
        const float s = 1.f / (1.f + expf(-zz)), sm = 1.f / (1.f + expf(zz));
        grad[k] = ((1.f - tt) * s - pw * tt * sm) / (float)n;
    }
    float out[1];
    block_sum<1>(acc, out);
    if (threadIdx.x == 0) part[blockIdx.x] = out[0];
}

__global__ void __launch_bounds__(256) k_bce_final(const float *__restrict__ part, int nparts, int64_t n,
                                                    float *__restrict__ loss)
{
    float acc[1] = {0.f};
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) acc[0] += part[k];
    float out[1];
    block_sum<1>(acc, out);
    if (threadIdx.x == 0) *loss = out[0] / (float)n;
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

unsigned grid_of(int64_t n, int per = 256, int cap = 152 * 16)
{
    int64_t b = (n + per - 1) / per;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}
}  // namespace

thread_local char g_nn_msg[256] = "";

dg_status nn_fail(dg_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_nn_msg, sizeof g_nn_msg, fmt, ap);
    va_end(ap);
    return st;
}

dg_status nn_done(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) return nn_fail(DG_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    g_nn_msg[0] = 0;
    return DG_OK;
}

namespace {

bool conv_shape_ok(int B, int Ci, int Co, int H, int W)
{
    return B > 0 && Ci > 0 && Co > 0 && H > 0 && W > 0 && Ci <= 4096 && Co <= 4096 &&
           (int64_t)B * ((std::max(Ci, Co) + 15) / 16) <= 65535 && (H + 15) / 16 <= 65535 &&
           (int64_t)H * W <= (int64_t)1 << 30 && (int64_t)B * Ci * H * W <= ((int64_t)1 << 40) &&
           (int64_t)B * Co * H * W <= ((int64_t)1 << 40) && (int64_t)Co * Ci <= ((int64_t)1 << 31) - 1;
}
}  // namespace

int64_t nn_conv_splits(int B, int Ci, int Co, int H, int W)
{
    const int64_t ctas = (int64_t)((Co + kDwO - 1) / kDwO) * Ci;
    const int64_t P = (int64_t)B * H * W;
    int64_t S = (152 * 4 + ctas - 1) / ctas;     // about four CTAs per SM
    S = std::min<int64_t>(S, std::max<int64_t>(1, P / 2048));
    return std::max<int64_t>(1, std::min<int64_t>(S, 1024));
}

int64_t nn_conv_scratch(int B, int Ci, int Co, int H, int W)
{
    return nn_conv_splits(B, Ci, Co, H, W) * ((int64_t)Co * Ci * 9 + Co);
}

cudaError_t launch_nn_conv_fwd(const float *x, const float *w, const float *b, float *y, int B, int Ci, int Co, int H,
                               int W, cudaStream_t s)
{
    const dim3 grid((W + kTW - 1) / kTW, (H + kTH - 1) / kTH, B * ((Co + kOC - 1) / kOC));
    k_conv3x3_tiled<false><<<grid, 128, 0, s>>>(x, w, b, y, Ci, Co, H, W);
    return cudaGetLastError();
}

cudaError_t launch_nn_conv_bwd(const float *x, const float *w, const float *dy, float *dx, float *dw, float *db, int B,
                               int Ci, int Co, int H, int W, float *scratch, cudaStream_t s)
{
    if (dx) {
        const dim3 grid((W + kTW - 1) / kTW, (H + kTH - 1) / kTH, B * ((Ci + kOC - 1) / kOC));
        k_conv3x3_tiled<true><<<grid, 128, 0, s>>>(dy, w, nullptr, dx, Co, Ci, H, W);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int S = (int)nn_conv_splits(B, Ci, Co, H, W);
    float *part = scratch, *part_b = scratch + (size_t)S * Co * Ci * 9;
    k_conv3x3_dw<<<dim3((Co + kDwO - 1) / kDwO, Ci, S), 256, 0, s>>>(x, dy, part, part_b, B, Ci, Co, H, W, S);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nw = (int64_t)Co * Ci * 9 + Co;
    k_conv3x3_dw_sum<<<(unsigned)std::min<int64_t>((nw + 255) / 256, 152 * 8), 256, 0, s>>>(part, part_b, dw, db, Co,
                                                                                             Ci, S);
    return cudaGetLastError();
}

cudaError_t launch_nn_relu(const float *z, const float *dh, float *out, int64_t n, cudaStream_t s)
{
    if (dh) k_relu_bwd<<<grid_of(n), 256, 0, s>>>(z, dh, out, n);
    else k_relu_fwd<<<grid_of(n), 256, 0, s>>>(z, out, n);
    return cudaGetLastError();
}

int nn_bce_parts(int64_t n) { return (int)grid_of(n, 256, 1024); }

cudaError_t launch_nn_bce(const float *z, const float *t, float pw, int64_t n, float *grad, float *part, float *loss,
                          cudaStream_t s)
{
    const int np = nn_bce_parts(n);
    k_bce<<<(unsigned)np, 256, 0, s>>>(z, t, pw, n, grad, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_bce_final<<<1, 256, 0, s>>>(part, np, n, loss);
    return cudaGetLastError();
}

cudaError_t launch_nn_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                           float eps, int step, cudaStream_t s)
{
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<grid_of(n), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace dg

extern "C" {

const char *dg_nn_last_error(void) { return dg::g_nn_msg; }

dg_status dg_nn_conv3x3_forward(const float *x, const float *w, const float *b, float *y, int32_t B, int32_t Ci,
                                int32_t Co, int32_t H, int32_t W, void *stream)
{
    if (!x || !w || !b || !y) return dg::nn_fail(DG_EINVAL, "dg_nn_conv3x3_forward: null pointer");
    if (!dg::conv_shape_ok(B, Ci, Co, H, W))
        return dg::nn_fail(DG_EINVAL, "dg_nn_conv3x3_forward: bad shape B=%d Ci=%d Co=%d H=%d W=%d", B, Ci, Co, H, W);
    return dg::nn_done(dg::launch_nn_conv_fwd(x, w, b, y, B, Ci, Co, H, W, (cudaStream_t)stream),
                       "dg_nn_conv3x3_forward");
}

int64_t dg_nn_conv3x3_scratch(int32_t B, int32_t Ci, int32_t Co, int32_t H, int32_t W)
{
    if (!dg::conv_shape_ok(B, Ci, Co, H, W)) return -1;
    return dg::nn_conv_scratch(B, Ci, Co, H, W);
}

dg_status dg_nn_conv3x3_backward(const float *x, const float *w, const float *dy, float *dx, float *dw, float *db,
                                 int32_t B, int32_t Ci, int32_t Co, int32_t H, int32_t W, float *scratch,
                                 void *stream)
{
    if (!x || !w || !dy || !dw || !db || !scratch)
        return dg::nn_fail(DG_EINVAL, "dg_nn_conv3x3_backward: null pointer");
    if (!dg::conv_shape_ok(B, Ci, Co, H, W))
        return dg::nn_fail(DG_EINVAL, "dg_nn_conv3x3_backward: bad shape B=%d Ci=%d Co=%d H=%d W=%d", B, Ci, Co, H,
                           W);
    return dg::nn_done(dg::launch_nn_conv_bwd(x, w, dy, dx, dw, db, B, Ci, Co, H, W, scratch, (cudaStream_t)stream),
                       "dg_nn_conv3x3_backward");
}

dg_status dg_nn_relu_forward(const float *z, float *h, int64_t n, void *stream)
{
    if (!z || !h || n < 0) return dg::nn_fail(DG_EINVAL, "dg_nn_relu_forward: null pointer or n < 0");
    if (n == 0) return DG_OK;
    return dg::nn_done(dg::launch_nn_relu(z, nullptr, h, n, (cudaStream_t)stream), "dg_nn_relu_forward");
}

dg_status dg_nn_relu_backward(const float *z, const float *dh, float *dz, int64_t n, void *stream)
{
    if (!z || !dh || !dz || n < 0) return dg::nn_fail(DG_EINVAL, "dg_nn_relu_backward: null pointer or n < 0");
    if (n == 0) return DG_OK;
    return dg::nn_done(dg::launch_nn_relu(z, dh, dz, n, (cudaStream_t)stream), "dg_nn_relu_backward");
}

int64_t dg_nn_bce_scratch(int64_t n) { return n > 0 ? dg::nn_bce_parts(n) : 0; }

dg_status dg_nn_bce_logits(const float *z, const float *t, float pos_weight, int64_t n, float *grad, float *loss,
                           float *scratch, void *stream)
{
    if (!z || !t || !grad || !loss || !scratch || n <= 0)
        return dg::nn_fail(DG_EINVAL, "dg_nn_bce_logits: null pointer or n <= 0");
    if (!(pos_weight > 0.f)) return dg::nn_fail(DG_EINVAL, "dg_nn_bce_logits: pos_weight must be > 0");
    return dg::nn_done(dg::launch_nn_bce(z, t, pos_weight, n, grad, scratch, loss, (cudaStream_t)stream),
                       "dg_nn_bce_logits");
}

dg_status dg_nn_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float beta1, float beta2,
                     float eps, int32_t step, void *stream)
{
    if (!p || !g || !m || !v || n < 0) return dg::nn_fail(DG_EINVAL, "dg_nn_adam: null pointer or n < 0");
    if (step < 1 || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return dg::nn_fail(DG_EINVAL, "dg_nn_adam: step %d, betas or eps out of range", step);
    if (n == 0) return DG_OK;
    return dg::nn_done(dg::launch_nn_adam(p, g, m, v, n, lr, beta1, beta2, eps, step, (cudaStream_t)stream),
                       "dg_nn_adam");
}

}  // extern "C"
