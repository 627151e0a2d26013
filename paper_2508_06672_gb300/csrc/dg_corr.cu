// dg_corr.cu -- direct position-domain correlation (Sec. III, Eq. 11).
//
// One CTA handles one tile of candidates (kWarps*R grid rows x 32 grid
// columns) for one snapshot k; R, the candidates (grid rows) per thread, is a
// launch choice (dg_options.rows, tuned by dg_autotune). Per candidate it computes the geometry
// (Eq. 3-10, FP64), then
//     C = sum_n y1[n] conj(y2~[n]) exp(j 2 pi nu n),
// y2~[n] = y2[n + L] (Eq. 9) or its 4-tap Lagrange interpolation at n + D,
// and writes |C|^2 (or |C|) into the snapshot's slice of the per-snapshot
// surface buffer; a separate pass sums the snapshots in order.
//
// Sum evaluation: y1 is staged in shared memory already multiplied by
// (-j)^n, which moves the wanted frequency to theta = 2 pi nu + pi/2. The
// sum over n of x[n] exp(j theta n) is then run as a second-order resonator
//     s[n] = x[n] + 2 cos(theta) s[n-1] - s[n-2],
//     sum  = exp(j theta (n_end-1)) (s[n_end-1] - exp(j theta) s[n_end-2]),
// with x[n] = y1'[n] conj(y2~[n]) folded into the same FMAs: 6 FMAs per
// candidate and sample, no per-sample phasor. Near theta = pi/2 the
// resonator is well conditioned (|nu| <= 0.2 is enforced). The closing phase
// is reduced in FP64.
//
// Shared memory holds a chunk of y1 (M samples) and the window of y2 that
// every candidate of the tile needs for that chunk (M + lag span + taps),
// converted to float/double; the captures stay L2-resident across CTAs.
#include <climits>

#include "dg_internal.cuh"

namespace dg {

template <typename T> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };

// M-sample chunks of y1 and a W-sample y2 window in shared memory.
template <typename T> struct Cfg;
template <> struct Cfg<float> { static constexpr int M = 2048, W = 4096; };
template <> struct Cfg<double> { static constexpr int M = 1024, W = 2048; };

__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }

template <typename C2> __device__ __forceinline__ C2 mk(double x, double y);
template <> __device__ __forceinline__ float2 mk<float2>(double x, double y) { return make_float2((float)x, (float)y); }
template <> __device__ __forceinline__ double2 mk<double2>(double x, double y) { return make_double2(x, y); }

template <typename T, int FMT>
__device__ __forceinline__ typename Cx<T>::t load_c(const void *b, int idx)
{
    const float2 v = IQ<FMT>::load(b, idx);
    return mk<typename Cx<T>::t>(v.x, v.y);
}

// Resonator update for two consecutive samples: (a0, b0) then (a1, b1).
// On entry s1 = s[n-1], s2 = s[n-2]; on exit s1 = s[n+1], s2 = s[n].
template <typename T, typename C2>
__device__ __forceinline__ void resonate2(const C2 &a0, const C2 &b0, const C2 &a1, const C2 &b1,
                                          T c2, C2 &s1, C2 &s2)
{
    // x = a * conj(b) = (a.x b.x + a.y b.y, a.y b.x - a.x b.y)
    s2.x = fma_(c2, s1.x, fma_(a0.y, b0.y, fma_(a0.x, b0.x, -s2.x)));
    s2.y = fma_(c2, s1.y, fma_(-a0.x, b0.y, fma_(a0.y, b0.x, -s2.y)));
    s1.x = fma_(c2, s2.x, fma_(a1.y, b1.y, fma_(a1.x, b1.x, -s1.x)));
    s1.y = fma_(c2, s2.y, fma_(-a1.x, b1.y, fma_(a1.y, b1.x, -s1.y)));
}

template <typename T, typename C2>
__device__ __forceinline__ C2 interp4(const C2 *q, const T *w)
{
    C2 r;
    r.x = fma_(w[3], q[3].x, fma_(w[2], q[2].x, fma_(w[1], q[1].x, w[0] * q[0].x)));
    r.y = fma_(w[3], q[3].y, fma_(w[2], q[2].y, fma_(w[1], q[1].y, w[0] * q[0].y)));
    return r;
}

// y2~ at sample n for lag L read straight from global memory (fallback when
// the tile's lag span does not fit the shared-memory window).
template <typename T, int FMT, int DELAY>
__device__ __forceinline__ typename Cx<T>::t y2_global(const void *y2, int N, int n, int L, const T *w)
{
    using C2 = typename Cx<T>::t;
    if constexpr (DELAY == DG_DELAY_INTEGER) {
        const int q = n + L;
        return (q >= 0 && q < N) ? load_c<T, FMT>(y2, q) : mk<C2>(0.0, 0.0);
    } else {
        C2 t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = n + L - 1 + u;
            t[u] = (q >= 0 && q < N) ? load_c<T, FMT>(y2, q) : mk<C2>(0.0, 0.0);
        }
        return interp4<T, C2>(t, w);
    }
}

template <typename T, int FMT, int DELAY, int R>
__global__ void __launch_bounds__(kThreads) k_corr_direct(CorrArgs a, int tiles_j)
{
    using C2 = typename Cx<T>::t;
    constexpr int MCH = Cfg<T>::M, WIN = Cfg<T>::W;
    constexpr int TAPS = (DELAY == DG_DELAY_LAGRANGE4) ? 3 : 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *y1s = reinterpret_cast<C2 *>(smem_raw);
    C2 *y2s = y1s + MCH;
    __shared__ int s_min[kWarps], s_max[kWarps];

    const int k = blockIdx.y;
    const int ti = blockIdx.x / tiles_j, tj = blockIdx.x % tiles_j;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // For each r the 32 lanes of a warp take a compact 4-row x 8-column patch
    // (warp w: columns 8 (w % 4) .. + 7 of the tile, rows 4R (w / 4) .. + 4R - 1;
    // lane: column lane % 8, row lane / 8, then 4 rows further per r). Their
    // lags then differ by at most 10 grid steps' worth, not 31 as along one
    // row, so the y2 window reads of a warp stay within a few banks' rows
    // where a grid step moves the lag by a sample or more.
    static_assert(kWarps == 8, "the lane mapping assumes 8 warps: 4 column blocks x 2 row blocks");
    const int j = tj * 32 + (warp & 3) * 8 + (lane & 7);
    const int row0 = ti * (kWarps * R) + (warp >> 2) * (4 * R) + (lane >> 3);
    const StepDesc sd = a.steps[k];
    const int N = sd.n;
    const int64_t G = a.G;

    double e[12];
#pragma unroll
    for (int t = 0; t < 12; ++t) e[t] = __ldg(a.eph + 12 * k + t);

    // ---- geometry of this thread's R candidates (FP64) ---------------------
    int off[R];
    T c2[R];
    T w[R][4];
    bool ok[R];
    int lmin = INT_MAX, lmax = INT_MIN;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = row0 + 4 * r;
        ok[r] = (i < a.nrows) && (j < a.nlon);
        off[r] = 0;
        c2[r] = (T)0;
        w[r][0] = (T)0; w[r][1] = (T)1; w[r][2] = (T)0; w[r][3] = (T)0;
        if (ok[r]) {
            const int64_t p = (int64_t)i * a.nlon + j;
            double D, nu;
            geometry(a.xyz[p], a.xyz[G + p], a.xyz[2 * G + p], e, a.fs, a.lambda, D, nu);
            if (!(fabs(nu) <= 0.2)) {
                atomicOr(a.err, ERR_NU_RANGE);
                ok[r] = false;
            } else if (!(fabs(D) < 1.0e9)) {
                atomicOr(a.err, ERR_LAG_RANGE);
                ok[r] = false;
            } else {
                const int L = lag_of(D, DELAY);
                off[r] = L;
                c2[r] = (T)(-2.0 * sinpi(2.0 * nu));
                if (DELAY == DG_DELAY_LAGRANGE4) {
                    const double mu = D - (double)L;
                    w[r][0] = (T)(-mu * (mu - 1.0) * (mu - 2.0) / 6.0);
                    w[r][1] = (T)((mu + 1.0) * (mu - 1.0) * (mu - 2.0) / 2.0);
                    w[r][2] = (T)(-(mu + 1.0) * mu * (mu - 2.0) / 2.0);
                    w[r][3] = (T)((mu + 1.0) * mu * (mu - 1.0) / 6.0);
                }
                lmin = min(lmin, L);
                lmax = max(lmax, L);
            }
        }
    }
    // ---- tile lag range --------------------------------------------------------
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        lmin = min(lmin, __shfl_xor_sync(0xffffffffu, lmin, d));
        lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, d));
    }
    if (lane == 0) {
        s_min[warp] = lmin;
        s_max[warp] = lmax;
    }
    __syncthreads();
    lmin = s_min[0];
    lmax = s_max[0];
#pragma unroll
    for (int u = 1; u < kWarps; ++u) {
        lmin = min(lmin, s_min[u]);
        lmax = max(lmax, s_max[u]);
    }
    if (lmin > lmax) return;  // no valid candidate in the tile (uniform)
    const int span = lmax - lmin;
    int mch = MCH;
    if (span + TAPS + MCH > WIN) mch = ((WIN - span - TAPS) / 64) * 64;
    const bool windowed = mch >= 64;
    if (!windowed) mch = MCH;
#pragma unroll
    for (int r = 0; r < R; ++r) off[r] = ok[r] ? off[r] - lmin : 0;

    C2 s1[R], s2[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        s1[r] = mk<C2>(0.0, 0.0);
        s2[r] = mk<C2>(0.0, 0.0);
    }

    // ---- sample loop -----------------------------------------------------------
    for (int n0 = 0; n0 < N; n0 += mch) {
        const int len = min(mch, N - n0);
        const int len2 = (len + 1) & ~1;
        __syncthreads();
        for (int q = threadIdx.x; q < len2; q += kThreads) {
            const int n = n0 + q;
            C2 v = (n < N) ? load_c<T, FMT>(sd.y1, n) : mk<C2>(0.0, 0.0);
            C2 o;
            switch (n & 3) {  // multiply by (-j)^n
            case 0: o = v; break;
            case 1: o.x = v.y; o.y = -v.x; break;
            case 2: o.x = -v.x; o.y = -v.y; break;
            default: o.x = -v.y; o.y = v.x; break;
            }
            y1s[q] = o;
        }
        if (windowed) {
            const int base = n0 + lmin - (TAPS ? 1 : 0);
            const int wl = len2 + span + TAPS;
            for (int q = threadIdx.x; q < wl; q += kThreads) {
                const int n = base + q;
                y2s[q] = (n >= 0 && n < N) ? load_c<T, FMT>(sd.y2, n) : mk<C2>(0.0, 0.0);
            }
        }
        __syncthreads();
        if (windowed) {
            if (DELAY == DG_DELAY_INTEGER) {
#pragma unroll 4
                for (int m = 0; m < len2; m += 2) {
                    const C2 a0 = y1s[m], a1 = y1s[m + 1];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const C2 *q = y2s + m + off[r];
                        resonate2<T, C2>(a0, q[0], a1, q[1], c2[r], s1[r], s2[r]);
                    }
                }
            } else {
#pragma unroll 2
                for (int m = 0; m < len2; m += 2) {
                    const C2 a0 = y1s[m], a1 = y1s[m + 1];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const C2 *q = y2s + m + off[r];
                        const C2 b0 = interp4<T, C2>(q, w[r]);
                        const C2 b1 = interp4<T, C2>(q + 1, w[r]);
                        resonate2<T, C2>(a0, b0, a1, b1, c2[r], s1[r], s2[r]);
                    }
                }
            }
        } else {
            for (int m = 0; m < len2; m += 2) {
                const C2 a0 = y1s[m], a1 = y1s[m + 1];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int L = off[r] + lmin;
                    const C2 b0 = y2_global<T, FMT, DELAY>(sd.y2, N, n0 + m, L, w[r]);
                    const C2 b1 = y2_global<T, FMT, DELAY>(sd.y2, N, n0 + m + 1, L, w[r]);
                    resonate2<T, C2>(a0, b0, a1, b1, c2[r], s1[r], s2[r]);
                }
            }
        }
    }

    // ---- close the resonators and write |C|^2 or |C| ---------------------------
    const int nend = (N + 1) & ~1;  // resonator steps taken (zero-padded to even)
    T *surf = reinterpret_cast<T *>(a.surf) + (int64_t)k * G;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (!ok[r]) continue;
        const int i = row0 + 4 * r;
        const int64_t p = (int64_t)i * a.nlon + j;
        double D, nu;
        geometry(a.xyz[p], a.xyz[G + p], a.xyz[2 * G + p], e, a.fs, a.lambda, D, nu);
        // E = exp(j theta (nend-1)) = exp(j 2 pi nu (nend-1)) * j^(nend-1)
        const double ph = nu * (double)(nend - 1);
        double se, ce;
        sincospi(2.0 * (ph - floor(ph)), &se, &ce);
        double ex, ey;
        switch ((nend - 1) & 3) {
        case 0: ex = ce; ey = se; break;
        case 1: ex = -se; ey = ce; break;
        case 2: ex = -ce; ey = -se; break;
        default: ex = se; ey = -ce; break;
        }
        // exp(j theta) = j exp(j 2 pi nu)
        double st, ct;
        sincospi(2.0 * nu, &st, &ct);
        const double thx = -st, thy = ct;
        const double ax = (double)s2[r].x, ay = (double)s2[r].y;
        const double ux = (double)s1[r].x - (thx * ax - thy * ay);
        const double uy = (double)s1[r].y - (thx * ay + thy * ax);
        const double cx = ex * ux - ey * uy;
        const double cy = ex * uy + ey * ux;
        const double pw = cx * cx + cy * cy;
        surf[p] = (T)((a.acc == DG_ACC_POWER) ? pw : sqrt(pw));
    }
}

template <typename T, int FMT, int DELAY, int R>
static cudaError_t launch_one(const CorrArgs &a, cudaStream_t s)
{
    using C2 = typename Cx<T>::t;
    const size_t smem = (size_t)(Cfg<T>::M + Cfg<T>::W) * sizeof(C2);
    // The attribute is per function and device; setting it each launch keeps
    // this correct for every device and thread at negligible cost.
    cudaError_t e = cudaFuncSetAttribute(k_corr_direct<T, FMT, DELAY, R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int tiles_i = (a.nrows + kWarps * R - 1) / (kWarps * R);
    const int tiles_j = (a.nlon + 31) / 32;
    const int64_t tiles = (int64_t)tiles_i * tiles_j;
    if (tiles > INT_MAX || a.K > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)tiles, (unsigned)a.K);
    k_corr_direct<T, FMT, DELAY, R><<<grid, kThreads, smem, s>>>(a, tiles_j);
    return cudaGetLastError();
}

// Grid rows per thread: FP32 4, 8 or 16; FP64 2 or 4. The defaults are the
// fastest measured on a 1001^2 grid (K = 50, N = 131072): FP32 8 with the
// integer delay (4 and 16 within 1 %), 4 with LAGRANGE4 (5 % ahead of 8).
template <typename T, int FMT, int DELAY>
static cudaError_t launch_rows(const CorrArgs &a, cudaStream_t s)
{
    if constexpr (sizeof(T) == 4) {
        const int rows = a.rows ? a.rows : (DELAY == DG_DELAY_INTEGER ? 8 : 4);
        switch (rows) {
        case 4: return launch_one<T, FMT, DELAY, 4>(a, s);
        case 8: return launch_one<T, FMT, DELAY, 8>(a, s);
        case 16: return launch_one<T, FMT, DELAY, 16>(a, s);
        default: return cudaErrorInvalidValue;
        }
    } else {
        switch (a.rows) {
        case 2: return launch_one<T, FMT, DELAY, 2>(a, s);
        case 0:
        case 4: return launch_one<T, FMT, DELAY, 4>(a, s);
        default: return cudaErrorInvalidValue;
        }
    }
}

template <typename T, int FMT>
static cudaError_t launch_delay(const CorrArgs &a, cudaStream_t s)
{
    return a.delay == DG_DELAY_INTEGER ? launch_rows<T, FMT, DG_DELAY_INTEGER>(a, s)
                                       : launch_rows<T, FMT, DG_DELAY_LAGRANGE4>(a, s);
}

template <typename T>
static cudaError_t launch_fmt(const CorrArgs &a, cudaStream_t s)
{
    switch (a.fmt) {
    case DG_IQ_C64: return launch_delay<T, DG_IQ_C64>(a, s);
    case DG_IQ_CI16: return launch_delay<T, DG_IQ_CI16>(a, s);
    case DG_IQ_CI8: return launch_delay<T, DG_IQ_CI8>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_corr_direct(const CorrArgs &a, cudaStream_t s)
{
    return a.prec == DG_PREC_FP64 ? launch_fmt<double>(a, s) : launch_fmt<float>(a, s);
}

}  // namespace dg
