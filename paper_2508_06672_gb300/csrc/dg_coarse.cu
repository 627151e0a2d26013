// dg_coarse.cu -- coarse delay-Doppler maps of each snapshot, back-projected
// onto the cells of the grid: the input of the learned proposal.
//
// Per snapshot k (captures y1, y2 of n samples; zero outside [0, n)):
//   X(l, nu) = sum_n y1[n] conj(y2[n + l]) e^{j 2 pi nu n}     (Eq. 11 at an
//   integer lag l and FDOA nu: the cross-ambiguity function of the two-step
//   TDOA/FDOA method, Sec. I), sampled at the lags l0 .. l0 + nlag - 1 that
//   the grid's nodes take (Eq. 9) and at Q bins nu_q = nu_lo + q delta over
//   the nodes' FDOA range [nu_lo, nu_hi] (Eq. 10).
// It is evaluated in chunks of M samples turned at the centre frequency
// nu_c = (nu_lo + nu_hi) / 2,
//   P_b(l) = sum_{m<M} y1[bM+m] e^{j 2 pi nu_c (bM+m)} conj(y2[bM+m+l]),
//   Xc(l, q) = sum_b e^{j 2 pi (nu_q - nu_c) b M} P_b(l),
// which is X(l, nu_q) with each sample's phase off by (nu_q - nu_c) m at most
// (M is chosen so that this stays below 1/8 cycle). A = |Xc|^2; mu = its mean.
// Cell (i, j), the quadrilateral of nodes (i, j) .. (i + 1, j + 1), gets the
// largest A / mu over the lags and bins its corners span (a max-pool of the
// map over the delay-Doppler box of the cell).
//
// Kernels:
//   k_coarse_init / k_coarse_geo / k_coarse_params   node lags and FDOAs
//       (double-float geometry, Eq. 3-10), their ranges per snapshot, the
//       map parameters;
//   k_caf_lags   the chunk sums: for one chunk and a tile of 896 lags, both
//       sample windows sit in shared memory; each thread slides a register
//       window of y2 across 7 consecutive lags (7 is odd, so the lanes'
//       strided reads hit distinct banks): 7 x 7 complex FMAs per 14 loads;
//   k_caf_bins   the chunk DFT at the Q bins and |.|^2, with the twiddles of
//       32 chunks staged in shared memory; deterministic partial sums of A;
//   k_caf_mean   mu per snapshot (fixed-order sum);
//   k_coarse_backproject   the max-pool per cell.
#include <climits>

#include "dg_internal.cuh"

namespace dg {
namespace {

constexpr int kCafR = 7;                          // lags per thread
constexpr int kCafThreads = 128;
constexpr int kCafTile = kCafR * kCafThreads;     // lags per k_caf_lags CTA
constexpr int kBinLags = 32;                      // lags per k_caf_bins CTA
constexpr int kBinChunks = 32;                    // chunks staged at a time

__device__ __forceinline__ float2 load_iq(const void *b, int fmt, int idx)
{
    if (fmt == DG_IQ_CI16) return IQ<DG_IQ_CI16>::load(b, idx);
    if (fmt == DG_IQ_CI8) return IQ<DG_IQ_CI8>::load(b, idx);
    return IQ<DG_IQ_C64>::load(b, idx);
}

// Order-preserving map of doubles onto unsigned 64-bit keys (and back).
__device__ __forceinline__ unsigned long long dkey(double x)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double undkey(unsigned long long k)
{
    const unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)u);
}

__global__ void k_coarse_init(int *lmm, unsigned long long *nmm, int K)
{
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        lmm[2 * k] = INT_MAX;
        lmm[2 * k + 1] = INT_MIN;
        nmm[2 * k] = ~0ull;
        nmm[2 * k + 1] = 0ull;
    }
}

// One thread per (node, snapshot k = blockIdx.y): Eq. 3-10 in double-float
// arithmetic on the FP32 pipes (ranges to about 1e-7 m), the lag of Eq. 9
// (round half away from zero; decided by the FP64 expression where D lies
// within 1e-6 of a rounding boundary) and the FDOA rounded to FP32; block
// minima / maxima, then one atomic per warp.
__global__ void __launch_bounds__(256) k_coarse_geo(CoarseArgs a)
{
    const int k = blockIdx.y;
    dfl ed[12];
#pragma unroll
    for (int t = 0; t < 12; ++t) ed[t] = {__ldg(a.ephf + 24 * k + 2 * t), __ldg(a.ephf + 24 * k + 2 * t + 1)};
    const dfl fsc = {a.fsc_hi, a.fsc_lo}, ilf = {a.ilf_hi, a.ilf_lo};
    int lmin = INT_MAX, lmax = INT_MIN;
    unsigned long long nmin = ~0ull, nmax = 0ull;
    const int64_t G = a.G;
    const float *xf = a.xyzf;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < G; p += (int64_t)gridDim.x * blockDim.x) {
        dfl D;
        float nu;
        geometry_df({xf[p], xf[G + p]}, {xf[2 * G + p], xf[3 * G + p]}, {xf[4 * G + p], xf[5 * G + p]}, ed, fsc, ilf,
                    D, nu);
        int L;
        if (!round_df(D, L)) {
            double e[12], D64, nu64;
            for (int t = 0; t < 12; ++t) e[t] = a.eph[12 * k + t];
            geometry(a.xyz[p], a.xyz[G + p], a.xyz[2 * G + p], e, a.fs, a.lambda, D64, nu64);
            L = lag_of(D64, DG_DELAY_INTEGER);
        }
        a.lag[k * G + p] = L;
        a.nu[k * G + p] = nu;
        lmin = min(lmin, L);
        lmax = max(lmax, L);
        const unsigned long long key = dkey((double)nu);
        nmin = min(nmin, key);
        nmax = max(nmax, key);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        lmin = min(lmin, __shfl_xor_sync(0xffffffffu, lmin, d));
        lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, d));
        nmin = min(nmin, __shfl_xor_sync(0xffffffffu, nmin, d));
        nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, d));
    }
    if ((threadIdx.x & 31) == 0 && lmin <= lmax) {
        atomicMin(a.lmm + 2 * k, lmin);
        atomicMax(a.lmm + 2 * k + 1, lmax);
        atomicMin(a.nmm + 2 * k, nmin);
        atomicMax(a.nmm + 2 * k + 1, nmax);
    }
}

__global__ void k_coarse_params(CoarseArgs a)
{
    for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
        const int l0 = a.lmm[2 * k], l1 = a.lmm[2 * k + 1];
        int nlag = (l1 >= l0) ? l1 - l0 + 1 : 0;
        if (nlag < 1 || nlag > a.nlag_cap) {
            atomicOr(a.err, ERR_LAG_RANGE);
            nlag = max(1, min(nlag, a.nlag_cap));
        }
        const double lo = undkey(a.nmm[2 * k]), hi = undkey(a.nmm[2 * k + 1]);
        CoarseStep s;
        s.l0 = l0;
        s.nlag = nlag;
        s.nu_lo = lo;
        s.delta = a.Q > 1 ? __ddiv_rn(__dsub_rn(hi, lo), (double)(a.Q - 1)) : 0.0;
        s.nu_c = __dmul_rn(0.5, __dadd_rn(lo, hi));
        s.mu = 0.0;
        a.st[k] = s;
    }
}

// Chunk sums P_b(l) for chunk b = blockIdx.y of snapshot k = blockIdx.z and
// the lags t0 .. t0 + 895 (t0 = 896 blockIdx.x, relative to l0).
__global__ void __launch_bounds__(kCafThreads) k_caf_lags(CoarseArgs a)
{
    extern __shared__ float2 sm[];
    const int k = blockIdx.z, b = blockIdx.y;
    const CoarseStep st = a.st[k];
    const StepDesc sd = a.steps[k];
    const int t0 = blockIdx.x * kCafTile;
    const int M = a.M;
    const int64_t s0 = (int64_t)b * M;
    if (t0 >= st.nlag || s0 >= sd.n) return;
    float2 *as = sm;                    // [M + R]   y1 turned at nu_c
    float2 *cs = sm + M + kCafR;        // [M + T + 2R] y2 from sample s0 + l0 + t0
    for (int m = threadIdx.x; m < M + kCafR; m += kCafThreads) {
        const int64_t n = s0 + m;
        float2 v = make_float2(0.f, 0.f);
        if (m < M && n < sd.n) {
            const float2 y = load_iq(sd.y1, sd.fmt, (int)n);
            double ph = __dmul_rn(st.nu_c, (double)n);
            ph = __dsub_rn(ph, floor(ph));
            float sn, cn;
            sincospif(2.0f * (float)ph, &sn, &cn);
            v = make_float2(y.x * cn - y.y * sn, y.x * sn + y.y * cn);
        }
        as[m] = v;
    }
    const int64_t c0 = s0 + st.l0 + t0;
    for (int i = threadIdx.x; i < M + kCafTile + 2 * kCafR; i += kCafThreads) {
        const int64_t n = c0 + i;
        cs[i] = (n >= 0 && n < sd.n) ? load_iq(sd.y2, sd.fmt, (int)n) : make_float2(0.f, 0.f);
    }
    __syncthreads();

    const int base = kCafR * threadIdx.x;
    float accr[kCafR], acci[kCafR], w1r[kCafR], w1i[kCafR], w2r[kCafR], w2i[kCafR];
#pragma unroll
    for (int r = 0; r < kCafR; ++r) {
        accr[r] = acci[r] = 0.f;
        const float2 v = cs[base + r];
        w1r[r] = v.x;
        w1i[r] = v.y;
    }
    for (int m0 = 0; m0 < M; m0 += kCafR) {
#pragma unroll
        for (int r = 0; r < kCafR; ++r) {
            const float2 v = cs[m0 + kCafR + base + r];
            w2r[r] = v.x;
            w2i[r] = v.y;
        }
#pragma unroll
        for (int s = 0; s < kCafR; ++s) {
            const float2 av = as[m0 + s];
#pragma unroll
            for (int r = 0; r < kCafR; ++r) {
                const int q = r + s;
                const float vr = q < kCafR ? w1r[q] : w2r[q - kCafR];
                const float vi = q < kCafR ? w1i[q] : w2i[q - kCafR];
                // av * conj(v)
                accr[r] = fmaf(av.x, vr, fmaf(av.y, vi, accr[r]));
                acci[r] = fmaf(av.y, vr, fmaf(-av.x, vi, acci[r]));
            }
        }
#pragma unroll
        for (int r = 0; r < kCafR; ++r) {
            w1r[r] = w2r[r];
            w1i[r] = w2i[r];
        }
    }
    float2 *Pk = a.P + ((size_t)k * a.nb_max + b) * a.nlag_cap;
#pragma unroll
    for (int r = 0; r < kCafR; ++r) {
        const int t = t0 + base + r;
        if (t < st.nlag) Pk[t] = make_float2(accr[r], acci[r]);
    }
}

// Xc at the Q bins for 32 lags of snapshot k = blockIdx.y; warp w takes the
// bins w, w + 8, ..., at most UQ of them (UQ >= Q / 8); A = |Xc|^2 and the
// block's sum of A (in a fixed order).
template <int UQ>
__global__ void __launch_bounds__(256) k_caf_bins(CoarseArgs a)
{
    extern __shared__ float2 sm[];
    __shared__ double red[8];
    const int k = blockIdx.y;
    const CoarseStep st = a.st[k];
    const int lt0 = blockIdx.x * kBinLags;
    const int ntb = gridDim.x;
    if (lt0 >= st.nlag) {
        if (threadIdx.x == 0) a.part[(size_t)k * ntb + blockIdx.x] = 0.0;
        return;
    }
    const int Q = a.Q, M = a.M;
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int nb = (a.steps[k].n + M - 1) / M;
    float2 *tw = sm;                       // [Q][32]
    float2 *ps = sm + Q * kBinChunks;      // [32 chunks][32 lags]
    float xr[UQ], xi[UQ];
#pragma unroll
    for (int u = 0; u < UQ; ++u) xr[u] = xi[u] = 0.f;
    for (int b0 = 0; b0 < nb; b0 += kBinChunks) {
        __syncthreads();
        for (int i = threadIdx.x; i < Q * kBinChunks; i += blockDim.x) {
            const int q = i / kBinChunks, b = b0 + i % kBinChunks;
            const double nq = __dadd_rn(st.nu_lo, __dmul_rn((double)q, st.delta));
            double ph = __dmul_rn(__dsub_rn(nq, st.nu_c), (double)b * (double)M);
            ph = __dsub_rn(ph, floor(ph));
            float sn, cn;
            sincospif(2.0f * (float)ph, &sn, &cn);
            tw[i] = make_float2(cn, sn);
        }
        for (int i = threadIdx.x; i < kBinChunks * kBinLags; i += blockDim.x) {
            const int b = b0 + i / kBinLags, t = lt0 + i % kBinLags;
            ps[i] = (b < nb && t < st.nlag) ? a.P[((size_t)k * a.nb_max + b) * a.nlag_cap + t] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int bb = 0; bb < kBinChunks; ++bb) {
            const float2 p = ps[bb * kBinLags + lane];
#pragma unroll
            for (int u = 0; u < UQ; ++u) {
                const int q = wq + 8 * u;
                if (q < Q) {
                    const float2 w = tw[q * kBinChunks + bb];
                    xr[u] = fmaf(w.x, p.x, fmaf(-w.y, p.y, xr[u]));
                    xi[u] = fmaf(w.x, p.y, fmaf(w.y, p.x, xi[u]));
                }
            }
        }
    }
    const int t = lt0 + lane;
    double sum = 0.0;
    if (t < st.nlag) {
        float *Ak = a.A + ((size_t)k * a.nlag_cap + t) * Q;
#pragma unroll
        for (int u = 0; u < UQ; ++u) {
            const int q = wq + 8 * u;
            if (q < Q) {
                const float v = fmaf(xr[u], xr[u], xi[u] * xi[u]);
                Ak[q] = v;
                sum += (double)v;
            }
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    if (lane == 0) red[wq] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        a.part[(size_t)k * ntb + blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(256) k_caf_mean(CoarseArgs a, int ntb)
{
    __shared__ double red[8];
    const int k = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < ntb; i += blockDim.x) s += a.part[(size_t)k * ntb + i];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        a.st[k].mu = t / ((double)a.st[k].nlag * (double)a.Q);
    }
}

// One thread per (cell, snapshot k = blockIdx.y).
__global__ void __launch_bounds__(256) k_coarse_backproject(CoarseArgs a)
{
    const int k = blockIdx.y;
    const CoarseStep st = a.st[k];
    const int Q = a.Q;
    const int nlon = a.nlon, ncol = nlon - 1;
    const int64_t ncell = (int64_t)(a.nlat - 1) * ncol;
    const int *lag = a.lag + (size_t)k * a.G;
    const float *nu = a.nu + (size_t)k * a.G;
    const float *Ak = a.A + (size_t)k * a.nlag_cap * Q;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = c / ncol, j = c % ncol;
        const int64_t p = i * nlon + j;
        const int64_t pc[4] = {p, p + 1, p + nlon, p + nlon + 1};
        int la = INT_MAX, lb = INT_MIN;
        double vmin = 1e300, vmax = -1e300;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            la = min(la, lag[pc[u]]);
            lb = max(lb, lag[pc[u]]);
            vmin = fmin(vmin, (double)nu[pc[u]]);
            vmax = fmax(vmax, (double)nu[pc[u]]);
        }
        la = max(0, la - st.l0);
        lb = min(st.nlag - 1, lb - st.l0);
        int qa = 0, qb = Q - 1;
        if (st.delta > 0.0) {
            qa = max(0, (int)floor(__ddiv_rn(__dsub_rn(vmin, st.nu_lo), st.delta)));
            qb = min(Q - 1, (int)ceil(__ddiv_rn(__dsub_rn(vmax, st.nu_lo), st.delta)));
        }
        float m = 0.f;
        for (int t = la; t <= lb; ++t)
            for (int q = qa; q <= qb; ++q) m = fmaxf(m, Ak[(size_t)t * Q + q]);
        a.maps[(size_t)k * ncell + c] = st.mu > 0.0 ? (float)((double)m / st.mu) : 0.f;
    }
}

unsigned blocks_for(int64_t n, int per, int cap)
{
    int64_t b = (n + per - 1) / per;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

int coarse_bin_tiles(int nlag_cap) { return (nlag_cap + kBinLags - 1) / kBinLags; }

cudaError_t launch_coarse(const CoarseArgs &a, cudaStream_t s, int *launches)
{
    cudaError_t e;
    k_coarse_init<<<1, 64, 0, s>>>(a.lmm, a.nmm, a.K);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_coarse_geo<<<dim3(blocks_for(a.G, 256, 152 * 4), a.K), 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_coarse_params<<<1, 64, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t lag_smem = sizeof(float2) * (2 * (size_t)a.M + kCafTile + 3 * kCafR);
    if (lag_smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k_caf_lags, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lag_smem);
        if (e != cudaSuccess) return e;
    }
    k_caf_lags<<<dim3((a.nlag_cap + kCafTile - 1) / kCafTile, a.nb_max, a.K), kCafThreads, lag_smem, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int ntb = coarse_bin_tiles(a.nlag_cap);
    const size_t bin_smem = sizeof(float2) * ((size_t)a.Q * kBinChunks + kBinChunks * kBinLags);
    const int uq = (a.Q + 7) / 8;
    auto bins = uq <= 1 ? k_caf_bins<1> : uq <= 2 ? k_caf_bins<2> : uq <= 4 ? k_caf_bins<4>
              : uq <= 8 ? k_caf_bins<8> : uq <= 16 ? k_caf_bins<16> : k_caf_bins<32>;
    if (bin_smem > 48 * 1024) {
        e = cudaFuncSetAttribute(bins, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bin_smem);
        if (e != cudaSuccess) return e;
    }
    bins<<<dim3(ntb, a.K), 256, bin_smem, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_caf_mean<<<a.K, 256, 0, s>>>(a, ntb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t ncell = (int64_t)(a.nlat - 1) * (a.nlon - 1);
    k_coarse_backproject<<<dim3(blocks_for(ncell, 256, 152 * 8), a.K), 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *launches += 7;
    return cudaSuccess;
}

}  // namespace dg
