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
// The network is small (tens of channels on a coarse map), so the kernels
// are direct: each thread of the convolutions produces one pixel for
// kOB output channels, reusing each input value kOB times from registers;
// the weight reductions are one CTA per (o, c) pair with a fixed-order tree,
// so every gradient is deterministic.
#include <cstdarg>
#include <cstdio>

#include "dg_internal.cuh"

namespace dg {

namespace {
constexpr int kOB = 8;  // output channels per thread (forward and data backward)

__global__ void __launch_bounds__(256) k_conv3x3_fwd(const float *__restrict__ x, const float *__restrict__ w,
                                                      const float *__restrict__ b, float *__restrict__ y, int B,
                                                      int Ci, int Co, int H, int W)
{
    const int nob = (Co + kOB - 1) / kOB;
    const int64_t total = (int64_t)B * nob * H * W;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t % W), i = (int)((t / W) % H);
        const int ob = (int)((t / ((int64_t)W * H)) % nob), n = (int)(t / ((int64_t)W * H * nob));
        const int o0 = ob * kOB;
        float acc[kOB];
#pragma unroll
        for (int k = 0; k < kOB; ++k) acc[k] = (o0 + k < Co) ? b[o0 + k] : 0.f;
        for (int c = 0; c < Ci; ++c) {
            const float *xc = x + ((size_t)n * Ci + c) * H * W;
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int ii = i + u - 1;
                if (ii < 0 || ii >= H) continue;
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const int jj = j + v - 1;
                    if (jj < 0 || jj >= W) continue;
                    const float xv = __ldg(xc + (size_t)ii * W + jj);
#pragma unroll
                    for (int k = 0; k < kOB; ++k)
                        if (o0 + k < Co) acc[k] = fmaf(__ldg(w + (((size_t)(o0 + k) * Ci + c) * 3 + u) * 3 + v), xv, acc[k]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kOB; ++k)
            if (o0 + k < Co) y[(((size_t)n * Co + o0 + k) * H + i) * W + j] = acc[k];
    }
}

// dx: the transposed convolution of dy with w (flipped taps, channels swapped)
__global__ void __launch_bounds__(256) k_conv3x3_bwd_data(const float *__restrict__ dy, const float *__restrict__ w,
                                                           float *__restrict__ dx, int B, int Ci, int Co, int H,
                                                           int W)
{
    const int ncb = (Ci + kOB - 1) / kOB;
    const int64_t total = (int64_t)B * ncb * H * W;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t % W), i = (int)((t / W) % H);
        const int cb = (int)((t / ((int64_t)W * H)) % ncb), n = (int)(t / ((int64_t)W * H * ncb));
        const int c0 = cb * kOB;
        float acc[kOB];
#pragma unroll
        for (int k = 0; k < kOB; ++k) acc[k] = 0.f;
        for (int o = 0; o < Co; ++o) {
            const float *dyo = dy + ((size_t)n * Co + o) * H * W;
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int ii = i - u + 1;
                if (ii < 0 || ii >= H) continue;
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const int jj = j - v + 1;
                    if (jj < 0 || jj >= W) continue;
                    const float g = __ldg(dyo + (size_t)ii * W + jj);
#pragma unroll
                    for (int k = 0; k < kOB; ++k)
                        if (c0 + k < Ci) acc[k] = fmaf(__ldg(w + (((size_t)o * Ci + c0 + k) * 3 + u) * 3 + v), g, acc[k]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kOB; ++k)
            if (c0 + k < Ci) dx[(((size_t)n * Ci + c0 + k) * H + i) * W + j] = acc[k];
    }
}

// Fixed-order block sum of 9 (or 1) values per thread: 256 threads.
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

// One CTA per (o, c): the 9 taps of dw[o, c]; the CTAs with c == 0 also
// give db[o].
__global__ void __launch_bounds__(256) k_conv3x3_bwd_weight(const float *__restrict__ x, const float *__restrict__ dy,
                                                             float *__restrict__ dw, float *__restrict__ db, int B,
                                                             int Ci, int Co, int H, int W)
{
    const int o = blockIdx.x / Ci, c = blockIdx.x % Ci;
    float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float accb[1] = {0.f};
    const int64_t HW = (int64_t)H * W;
    for (int n = 0; n < B; ++n) {
        const float *dyo = dy + ((size_t)n * Co + o) * HW;
        const float *xc = x + ((size_t)n * Ci + c) * HW;
        for (int64_t p = threadIdx.x; p < HW; p += blockDim.x) {
            const int i = (int)(p / W), j = (int)(p % W);
            const float g = __ldg(dyo + p);
            if (c == 0) accb[0] += g;
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int ii = i + u - 1;
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const int jj = j + v - 1;
                    const float xv = (ii >= 0 && ii < H && jj >= 0 && jj < W) ? __ldg(xc + (size_t)ii * W + jj) : 0.f;
                    acc[3 * u + v] = fmaf(g, xv, acc[3 * u + v]);
                }
            }
        }
    }
    float out[9];
    block_sum<9>(acc, out);
    if (threadIdx.x == 0)
        for (int k = 0; k < 9; ++k) dw[((size_t)o * Ci + c) * 9 + k] = out[k];
    if (c == 0) {
        __syncthreads();
        float ob[1];
        block_sum<1>(accb, ob);
        if (threadIdx.x == 0) db[o] = ob[0];
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

namespace {
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

bool conv_shape_ok(int B, int Ci, int Co, int H, int W)
{
    return B > 0 && Ci > 0 && Co > 0 && H > 0 && W > 0 && Ci <= 4096 && Co <= 4096 &&
           (int64_t)H * W <= (int64_t)1 << 30 && (int64_t)B * Ci * H * W <= ((int64_t)1 << 40) &&
           (int64_t)B * Co * H * W <= ((int64_t)1 << 40) && (int64_t)Co * Ci <= ((int64_t)1 << 31) - 1;
}
}  // namespace

cudaError_t launch_nn_conv_fwd(const float *x, const float *w, const float *b, float *y, int B, int Ci, int Co, int H,
                               int W, cudaStream_t s)
{
    const int64_t total = (int64_t)B * ((Co + kOB - 1) / kOB) * H * W;
    k_conv3x3_fwd<<<grid_of(total), 256, 0, s>>>(x, w, b, y, B, Ci, Co, H, W);
    return cudaGetLastError();
}

cudaError_t launch_nn_conv_bwd(const float *x, const float *w, const float *dy, float *dx, float *dw, float *db, int B,
                               int Ci, int Co, int H, int W, cudaStream_t s)
{
    if (dx) {
        const int64_t total = (int64_t)B * ((Ci + kOB - 1) / kOB) * H * W;
        k_conv3x3_bwd_data<<<grid_of(total), 256, 0, s>>>(dy, w, dx, B, Ci, Co, H, W);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_conv3x3_bwd_weight<<<(unsigned)(Co * Ci), 256, 0, s>>>(x, dy, dw, db, B, Ci, Co, H, W);
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

dg_status dg_nn_conv3x3_backward(const float *x, const float *w, const float *dy, float *dx, float *dw, float *db,
                                 int32_t B, int32_t Ci, int32_t Co, int32_t H, int32_t W, void *stream)
{
    if (!x || !w || !dy || !dw || !db) return dg::nn_fail(DG_EINVAL, "dg_nn_conv3x3_backward: null pointer");
    if (!dg::conv_shape_ok(B, Ci, Co, H, W))
        return dg::nn_fail(DG_EINVAL, "dg_nn_conv3x3_backward: bad shape B=%d Ci=%d Co=%d H=%d W=%d", B, Ci, Co, H,
                           W);
    return dg::nn_done(dg::launch_nn_conv_bwd(x, w, dy, dx, dw, db, B, Ci, Co, H, W, (cudaStream_t)stream),
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
