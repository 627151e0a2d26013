// dg_cdft.cu -- Eq. 11 evaluated per integer lag as a chunked DFT.
//
// For one snapshot, every candidate c has an integer lag L_c (Eq. 9) and a
// normalised FDOA nu_c = dfreq / fs (Eq. 10). All candidates with the same L
// share the lag product z_L[n] = y1[n] conj(y2[n + L]), so
//     C_c = sum_n z_L[n] e^{j 2 pi nu_c n}
//         = sum_b e^{j 2 pi nu_c b M} W_b(nu_c),
//     W_b(nu) = sum_{m<M} z_L[bM + m] e^{j 2 pi nu m}        (chunk b, M samples).
// W_b is a smooth function of nu (its spectral width is ~1/M), and the FDOAs
// that share one lag span a narrow band [nu_lo(L), nu_hi(L)], so W_b is
// evaluated once per lag on Q = 64 bins nu_lo + q * Delta (a dense [chunks x
// M] x [M x Q] contraction) and each candidate interpolates linearly between
// the two bins around its own nu_c. Delta is the widest per-lag span of the
// snapshot divided by Q - 1; with the spans of LEO geometry (< 1e-4 cycles
// per sample) M * Delta < 1e-3 and the interpolation error is ~(pi M Delta)^2/8.
//
// Pipeline per snapshot: lag range (all snapshots at once) -> histogram of
// lags with each lag's FDOA range -> scan (bucket offsets, bin spacing) ->
// scatter of candidate indices into lag buckets -> contraction W[L][b][q] ->
// per-candidate combine into the snapshot's surface slice.
#include <climits>

#include "dg_internal.cuh"

namespace dg {

// Order-preserving map of doubles to unsigned 64-bit keys (for atomic min/max).
__device__ __forceinline__ unsigned long long okey(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double unokey(unsigned long long k)
{
    return __longlong_as_double((long long)((k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k));
}

__device__ __forceinline__ void load_eph(const double *p, double e[12])
{
#pragma unroll
    for (int t = 0; t < 12; ++t) e[t] = __ldg(p + t);
}

// ---------------------------------------------------------------------------
// 1. Lag range of every snapshot: lr[k] = {min L, max L} (init INT_MAX/INT_MIN).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_cdft_range(const double *__restrict__ xyz, const double *__restrict__ eph,
                                                    int64_t G, double fs, double lambda, int *lr, unsigned *err)
{
    __shared__ int smin[8], smax[8];
    const int k = blockIdx.y;
    double e[12];
    load_eph(eph + 12 * (size_t)k, e);
    int lo = INT_MAX, hi = INT_MIN;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < G; p += (int64_t)gridDim.x * blockDim.x) {
        double D, nu;
        geometry(xyz[p], xyz[G + p], xyz[2 * G + p], e, fs, lambda, D, nu);
        if (!(fabs(D) < 1.0e9)) {
            atomicOr(err, ERR_LAG_RANGE);
            continue;
        }
        const int L = (int)round(D);
        lo = min(lo, L);
        hi = max(hi, L);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, d));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, d));
    }
    if ((threadIdx.x & 31) == 0) {
        smin[threadIdx.x >> 5] = lo;
        smax[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lo = min(lo, smin[w]);
            hi = max(hi, smax[w]);
        }
        if (lo <= hi) {
            atomicMin(lr + 2 * k, lo);
            atomicMax(lr + 2 * k + 1, hi);
        }
    }
}

__global__ void k_cdft_range_init(int *lr, int K)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < K) {
        lr[2 * k] = INT_MAX;
        lr[2 * k + 1] = INT_MIN;
    }
}

// ---------------------------------------------------------------------------
// 2. Histogram of lags and each lag's FDOA range (one snapshot).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_cdft_hist(const double *__restrict__ xyz, const double *__restrict__ eph_k,
                                                   int64_t G, double fs, double lambda, const int *lr_k,
                                                   int *candB, double *candNu, int *count,
                                                   unsigned long long *nulo, unsigned long long *nuhi)
{
    double e[12];
    load_eph(eph_k, e);
    const int lmin = lr_k[0];
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < G; p += (int64_t)gridDim.x * blockDim.x) {
        double D, nu;
        geometry(xyz[p], xyz[G + p], xyz[2 * G + p], e, fs, lambda, D, nu);
        if (!(fabs(D) < 1.0e9)) {
            candB[p] = -1;
            continue;
        }
        const int b = (int)round(D) - lmin;
        candB[p] = b;
        candNu[p] = nu;
        atomicAdd(count + b, 1);
        const unsigned long long key = okey(nu);
        atomicMin(nulo + b, key);
        atomicMax(nuhi + b, key);
    }
}

// ---------------------------------------------------------------------------
// 3. Scan (one CTA of 1024 threads): bucket offsets, combine-group offsets
//    (groups of kCombineThreads candidates never straddle buckets), the
//    per-bucket lowest FDOA as a double, and the bin spacing of the snapshot.
// ---------------------------------------------------------------------------
constexpr int kCombineThreads = 256;

__global__ void __launch_bounds__(1024) k_cdft_scan(int NB, const int *count, const unsigned long long *nulo,
                                                    const unsigned long long *nuhi, int *offs, int *gofs,
                                                    double *nulo_d, double *delta, int Q)
{
    __shared__ int s_c[1024], s_g[1024];
    __shared__ double s_span[32];
    const int t = threadIdx.x;
    const int per = (NB + 1023) / 1024;
    const int b0 = min(NB, t * per), b1 = min(NB, b0 + per);
    int c = 0, g = 0;
    double span = 0.0;
    for (int b = b0; b < b1; ++b) {
        const int n = count[b];
        c += n;
        g += (n + kCombineThreads - 1) / kCombineThreads;
        if (n > 0) {
            const double lo = unokey(nulo[b]), hi = unokey(nuhi[b]);
            nulo_d[b] = lo;
            span = fmax(span, hi - lo);
        } else {
            nulo_d[b] = 0.0;
        }
    }
    s_c[t] = c;
    s_g[t] = g;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) span = fmax(span, __shfl_xor_sync(0xffffffffu, span, d));
    if ((t & 31) == 0) s_span[t >> 5] = span;
    __syncthreads();
    // inclusive Hillis-Steele scan over the 1024 per-thread totals
    for (int d = 1; d < 1024; d <<= 1) {
        const int vc = t >= d ? s_c[t - d] : 0, vg = t >= d ? s_g[t - d] : 0;
        __syncthreads();
        s_c[t] += vc;
        s_g[t] += vg;
        __syncthreads();
    }
    int oc = t ? s_c[t - 1] : 0, og = t ? s_g[t - 1] : 0;
    for (int b = b0; b < b1; ++b) {
        offs[b] = oc;
        gofs[b] = og;
        const int n = count[b];
        oc += n;
        og += (n + kCombineThreads - 1) / kCombineThreads;
    }
    if (t == 1023) {
        offs[NB] = s_c[1023];
        gofs[NB] = s_g[1023];
    }
    if (t == 0) {
        double m = 0.0;
        for (int w = 0; w < 32; ++w) m = fmax(m, s_span[w]);
        // bins must cover [nu_lo, nu_lo + span]; keep Delta > 0 for single-FDOA lags
        *delta = fmax(m / (double)(Q - 1), 1e-15);
    }
}

// ---------------------------------------------------------------------------
// 4. Scatter candidate indices into their lag buckets (order inside a bucket
//    is arbitrary; each candidate's result does not depend on it).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_cdft_scatter(int64_t G, const int *candB, const int *offs, int *cursor,
                                                      int *order)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < G; p += (int64_t)gridDim.x * blockDim.x) {
        const int b = candB[p];
        if (b < 0) continue;
        order[offs[b] + atomicAdd(cursor + b, 1)] = (int)p;
    }
}

// ---------------------------------------------------------------------------
// 5. Contraction on CUDA cores (FP32): W[bucket][chunk][q] for 16 chunks per
//    CTA. Thread (q, s) keeps 4 chunks' accumulators for bin q; the bin's
//    phasor e^{j 2 pi (nu_lo + q Delta) m} runs by recurrence, restarted
//    exactly (FP64-reduced phase) every 64 samples.
// ---------------------------------------------------------------------------
constexpr int kCG = 16;     // chunks per contraction CTA
constexpr int kSub = 256;   // samples staged per pass

template <int FMT>
__global__ void __launch_bounds__(256) k_cdft_contract_f32(const StepDesc *__restrict__ sd_k, const int *lr_k,
                                                           const int *count, const double *nulo_d, const double *delta,
                                                           int M, int B, float2 *__restrict__ W)
{
    __shared__ float2 zs[kSub][kCG];
    const int b = blockIdx.x;
    if (count[b] == 0) return;
    const int c0 = blockIdx.y * kCG;
    const StepDesc sd = *sd_k;
    const int N = sd.n;
    const int L = lr_k[0] + b;
    const int q = threadIdx.x & 63, s = threadIdx.x >> 6;
    const double fq = nulo_d[b] + (double)q * (*delta);
    float sf, cf;
    {
        double st, ct;
        sincospi(2.0 * (fq - floor(fq)), &st, &ct);
        sf = (float)st;
        cf = (float)ct;
    }
    float2 acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = make_float2(0.f, 0.f);
    for (int m0 = 0; m0 < M; m0 += kSub) {
        __syncthreads();
        for (int i = threadIdx.x; i < kSub * kCG; i += blockDim.x) {
            const int cc = i / kSub, m = i % kSub;
            const int n = (c0 + cc) * M + m0 + m, n2 = n + L;
            float2 z = make_float2(0.f, 0.f);
            if (c0 + cc < B && m0 + m < M && n < N && n2 >= 0 && n2 < N) {
                const float2 a = IQ<FMT>::load(sd.y1, n), bb = IQ<FMT>::load(sd.y2, n2);
                z.x = fmaf(a.x, bb.x, a.y * bb.y);
                z.y = fmaf(a.y, bb.x, -a.x * bb.y);
            }
            zs[m][cc] = z;
        }
        __syncthreads();
        const int mlen = min(kSub, M - m0);
        for (int mm = 0; mm < mlen; mm += 64) {
            // exact phasor at sample m0 + mm of the chunk
            float px, py;
            {
                const double ph = fq * (double)(m0 + mm);
                double st, ct;
                sincospi(2.0 * (ph - floor(ph)), &st, &ct);
                px = (float)ct;
                py = (float)st;
            }
            const int mend = min(mm + 64, mlen);
            for (int m = mm; m < mend; ++m) {
                const float4 z01 = *reinterpret_cast<const float4 *>(&zs[m][4 * s]);
                const float4 z23 = *reinterpret_cast<const float4 *>(&zs[m][4 * s + 2]);
                acc[0].x = fmaf(z01.x, px, fmaf(-z01.y, py, acc[0].x));
                acc[0].y = fmaf(z01.x, py, fmaf(z01.y, px, acc[0].y));
                acc[1].x = fmaf(z01.z, px, fmaf(-z01.w, py, acc[1].x));
                acc[1].y = fmaf(z01.z, py, fmaf(z01.w, px, acc[1].y));
                acc[2].x = fmaf(z23.x, px, fmaf(-z23.y, py, acc[2].x));
                acc[2].y = fmaf(z23.x, py, fmaf(z23.y, px, acc[2].y));
                acc[3].x = fmaf(z23.z, px, fmaf(-z23.w, py, acc[3].x));
                acc[3].y = fmaf(z23.z, py, fmaf(z23.w, px, acc[3].y));
                const float nx = fmaf(px, cf, -py * sf);
                py = fmaf(px, sf, py * cf);
                px = nx;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int ch = c0 + 4 * s + u;
        if (ch < B) W[((size_t)b * B + ch) * 64 + q] = acc[u];
    }
}

// ---------------------------------------------------------------------------
// 6. Combine: one thread per candidate, kCombineThreads candidates of one
//    bucket per CTA; W of the bucket streams through shared memory in
//    segments of kSeg chunks.
// ---------------------------------------------------------------------------
constexpr int kSeg = 32;

template <typename T>
__global__ void __launch_bounds__(kCombineThreads) k_cdft_combine(int NB, const int *count, const int *offs,
                                                                  const int *gofs, const int *order,
                                                                  const double *candNu, const double *nulo_d,
                                                                  const double *delta, const float2 *__restrict__ W,
                                                                  int M, int B, int acc_mode, T *surf_k)
{
    __shared__ float2 ws[kSeg][64];
    const int gid = blockIdx.x;
    if (gid >= gofs[NB]) return;
    int lo = 0, hi = NB - 1;  // bucket b with gofs[b] <= gid < gofs[b+1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (gofs[mid] <= gid) lo = mid; else hi = mid - 1;
    }
    const int b = lo;
    const int j = (gid - gofs[b]) * kCombineThreads + threadIdx.x;
    const bool active = j < count[b];
    const int c = active ? order[offs[b] + j] : 0;
    const double nu = active ? candNu[c] : nulo_d[b];
    const double u = (nu - nulo_d[b]) / (*delta);
    int q0 = (int)floor(u);
    q0 = max(0, min(62, q0));
    const float t = (float)(u - (double)q0);
    const float w0 = 1.f - t, w1 = t;
    // e^{j 2 pi nu M}: chunk-to-chunk phase step
    float ex, ey;
    {
        const double ph = nu * (double)M;
        double st, ct;
        sincospi(2.0 * (ph - floor(ph)), &st, &ct);
        ex = (float)ct;
        ey = (float)st;
    }
    float cx = 0.f, cy = 0.f, px = 1.f, py = 0.f;
    const float2 *Wb = W + (size_t)b * B * 64;
    for (int s0 = 0; s0 < B; s0 += kSeg) {
        const int slen = min(kSeg, B - s0);
        __syncthreads();
        for (int i = threadIdx.x; i < slen * 64; i += kCombineThreads) ws[i >> 6][i & 63] = Wb[(size_t)s0 * 64 + i];
        __syncthreads();
        // exact chunk phase at the segment start
        {
            const double ph = nu * (double)s0 * (double)M;
            double st, ct;
            sincospi(2.0 * (ph - floor(ph)), &st, &ct);
            px = (float)ct;
            py = (float)st;
        }
        for (int i = 0; i < slen; ++i) {
            const float2 a = ws[i][q0], bb = ws[i][q0 + 1];
            const float zx = fmaf(w0, a.x, w1 * bb.x), zy = fmaf(w0, a.y, w1 * bb.y);
            cx = fmaf(px, zx, fmaf(-py, zy, cx));
            cy = fmaf(px, zy, fmaf(py, zx, cy));
            const float nx = fmaf(px, ex, -py * ey);
            py = fmaf(px, ey, py * ex);
            px = nx;
        }
    }
    if (active) {
        const double pw = (double)cx * cx + (double)cy * cy;
        surf_k[c] = (T)(acc_mode == DG_ACC_POWER ? pw : sqrt(pw));
    }
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
static unsigned grid_for(int64_t n, int per)
{
    int64_t b = (n + per - 1) / per;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_cdft_range(const double *xyz, const double *eph, int K, int64_t G, double fs, double lambda,
                              int *lr, unsigned *err, cudaStream_t s)
{
    k_cdft_range_init<<<(K + 127) / 128, 128, 0, s>>>(lr, K);
    dim3 grid(grid_for(G, 256 * 4), (unsigned)K);
    k_cdft_range<<<grid, 256, 0, s>>>(xyz, eph, G, fs, lambda, lr, err);
    return cudaGetLastError();
}

cudaError_t launch_cdft_plan(const CdftStepArgs &a, cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(a.count, 0, sizeof(int) * (size_t)a.NB, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.cursor, 0, sizeof(int) * (size_t)a.NB, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.nulo, 0xff, sizeof(unsigned long long) * (size_t)a.NB, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.nuhi, 0, sizeof(unsigned long long) * (size_t)a.NB, s)) != cudaSuccess) return e;
    k_cdft_hist<<<grid_for(a.G, 256), 256, 0, s>>>(a.xyz, a.eph_k, a.G, a.fs, a.lambda, a.lr_k, a.candB, a.candNu,
                                                    a.count, a.nulo, a.nuhi);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_cdft_scan<<<1, 1024, 0, s>>>(a.NB, a.count, a.nulo, a.nuhi, a.offs, a.gofs, a.nulo_d, a.delta, 64);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_cdft_scatter<<<grid_for(a.G, 256), 256, 0, s>>>(a.G, a.candB, a.offs, a.cursor, a.order);
    return cudaGetLastError();
}

cudaError_t launch_cdft_contract(const CdftStepArgs &a, cudaStream_t s)
{
    dim3 cg((unsigned)a.NB, (unsigned)((a.B + kCG - 1) / kCG));
    switch (a.fmt) {
    case DG_IQ_C64:
        k_cdft_contract_f32<DG_IQ_C64><<<cg, 256, 0, s>>>(a.sd_k, a.lr_k, a.count, a.nulo_d, a.delta, a.M, a.B, a.W);
        break;
    case DG_IQ_CI16:
        k_cdft_contract_f32<DG_IQ_CI16><<<cg, 256, 0, s>>>(a.sd_k, a.lr_k, a.count, a.nulo_d, a.delta, a.M, a.B, a.W);
        break;
    default:
        k_cdft_contract_f32<DG_IQ_CI8><<<cg, 256, 0, s>>>(a.sd_k, a.lr_k, a.count, a.nulo_d, a.delta, a.M, a.B, a.W);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_cdft_combine(const CdftStepArgs &a, cudaStream_t s)
{
    // an upper bound on the number of groups: G / 256 + one partial group per bucket
    const int64_t groups = a.G / kCombineThreads + a.NB + 1;
    k_cdft_combine<float><<<(unsigned)groups, kCombineThreads, 0, s>>>(
        a.NB, a.count, a.offs, a.gofs, a.order, a.candNu, a.nulo_d, a.delta, a.W, a.M, a.B, a.acc,
        reinterpret_cast<float *>(a.surf_k));
    return cudaGetLastError();
}

}  // namespace dg
