// dg_cdft.cu -- Eq. 11 evaluated per integer lag as a chunked DFT.
//
// For one snapshot, every candidate c has an integer lag L_c (Eq. 9) and a
// normalised FDOA nu_c = dfreq / fs (Eq. 10). All candidates with the same L
// share the lag product z_L[n] = y1[n] conj(y2[n + L]), so
//     C_c = sum_n z_L[n] e^{j 2 pi nu_c n}
//         = sum_b e^{j 2 pi nu_c b M} W_b(nu_c),
//     W_b(nu) = sum_{m<M} z_L[bM + m] e^{j 2 pi nu m}          (chunk b).
// W_b is smooth in nu (spectral width ~1/M) and the FDOAs of one snapshot
// span a narrow band [nu_min, nu_max] (LEO geometry: < 2e-4 cycles/sample),
// so W_b is evaluated once per (lag, chunk) on Q = 64 bins
// nu_q = nu_min + (q - 2) Delta, Delta = (nu_max - nu_min) / 59 (two bins of
// padding on each side) -- a dense [lag x chunk rows] x [M] x [64 bins]
// contraction whose DFT matrix V[m][q] = e^{j 2 pi nu_q m} is shared by every
// row of the snapshot -- and each candidate interpolates between the six
// bins around its own FDOA (Lagrange, nodes q0 - 2 .. q0 + 3 with the FDOA
// between q0 and q0 + 1). The interpolation error is at most about
// 4.9e-3 (2 pi M Delta)^6 of the coherent sum; the snapshot is rejected
// (DG_EUNSUPPORTED) if M * Delta > kCdftMDelta.
//
// All snapshots of a batch are processed by the same launches:
//   geo      FP64 geometry once per (candidate, snapshot): lag and FDOA kept,
//            per-snapshot lag and FDOA ranges by atomics (the host sizes the
//            buckets from the lag range);
//   hist     count per (snapshot, lag) bucket, aggregated in shared memory;
//   scan     one CTA per snapshot: bucket offsets, combine-group offsets and
//            the snapshot's bins;
//   scatter  candidate indices sorted by bucket (grouped by grid tile
//            within), and their FDOAs in the same order;
//   contract W[bucket][chunk] = 64 bins, stored planar (64 real parts then 64
//            imaginary parts); FP32 CUDA cores here, tensor cores in
//            dg_cdft_mma.cu;
//   combine  one thread per candidate: interpolate, rotate by the chunk's
//            FDOA phase, sum over chunks, |C|^2 or |C| into the surface.
#include <climits>

#include "dg_internal.cuh"

namespace dg {

__device__ __forceinline__ unsigned fkey(float x)
{
    const unsigned b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float unfkey(unsigned k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Step of the batch that owns global bucket b (bbase[s] <= b < bbase[s+1]).
__device__ __forceinline__ int step_of(const int *base, int S, int b)
{
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// geo: lag and FDOA of every (candidate, snapshot), lag range per snapshot.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 4) k_cdft_geo(CdftBatch a)
{
    __shared__ int smin[8], smax[8];
    const int s = blockIdx.y;
    dfl ed[12];
#pragma unroll
    for (int t = 0; t < 12; ++t) ed[t] = {__ldg(a.ephf + 24 * (size_t)s + 2 * t), __ldg(a.ephf + 24 * (size_t)s + 2 * t + 1)};
    const dfl fsc = {a.fsc_hi, a.fsc_lo};
    __shared__ unsigned sflo[8], sfhi[8];
    int lo = INT_MAX, hi = INT_MIN;
    unsigned flo = 0xffffffffu, fhi = 0u;
    const float *xf = a.xyzf;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.G; p += (int64_t)gridDim.x * blockDim.x) {
        // double-float geometry; the lag is decided by the FP64 expression
        // (the oracle's) only when D lies within 1e-6 of a rounding boundary
        dfl D;
        float nuf;
        geometry_df({xf[p], xf[a.G + p]}, {xf[2 * a.G + p], xf[3 * a.G + p]}, {xf[4 * a.G + p], xf[5 * a.G + p]},
                    ed, fsc, {a.ilf_hi, a.ilf_lo}, D, nuf);
        int L = INT_MIN;
        float mu = 0.f;
        bool ok = fabsf(D.hi) < 1.0e9f;
        if (ok && !(a.delay == DG_DELAY_INTEGER ? round_df(D, L) : floor_df(D, L, mu))) {
            double e[12], D64, nu64;
            for (int t = 0; t < 12; ++t) e[t] = a.eph[12 * (size_t)s + t];
            geometry(a.xyz[p], a.xyz[a.G + p], a.xyz[2 * a.G + p], e, a.fs, a.lambda, D64, nu64);
            ok = fabs(D64) < 1.0e9;
            if (ok) {
                L = lag_of(D64, a.delay);
                mu = (float)(D64 - (double)L);
            }
        }
        if (ok) {
            // Lagrange4 also needs the lags L - 1 and L + 2 of the stencil
            lo = min(lo, a.delay == DG_DELAY_INTEGER ? L : L - 1);
            hi = max(hi, a.delay == DG_DELAY_INTEGER ? L : L + 2);
            flo = min(flo, fkey(nuf));
            fhi = max(fhi, fkey(nuf));
        } else {
            atomicOr(a.err, ERR_LAG_RANGE);
        }
        a.candL[(size_t)s * a.G + p] = L;
        a.candNu[(size_t)s * a.G + p] = nuf;
        if (a.delay != DG_DELAY_INTEGER) a.candMu[(size_t)s * a.G + p] = mu;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, d));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, d));
        flo = min(flo, __shfl_xor_sync(0xffffffffu, flo, d));
        fhi = max(fhi, __shfl_xor_sync(0xffffffffu, fhi, d));
    }
    if ((threadIdx.x & 31) == 0) {
        smin[threadIdx.x >> 5] = lo;
        smax[threadIdx.x >> 5] = hi;
        sflo[threadIdx.x >> 5] = flo;
        sfhi[threadIdx.x >> 5] = fhi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) {
            lo = min(lo, smin[w]);
            hi = max(hi, smax[w]);
            flo = min(flo, sflo[w]);
            fhi = max(fhi, sfhi[w]);
        }
        if (lo <= hi) {
            atomicMin(a.lr + 2 * s, lo);
            atomicMax(a.lr + 2 * s + 1, hi);
            atomicMin(a.nur + 2 * s, flo);
            atomicMax(a.nur + 2 * s + 1, fhi);
        }
    }
}

__global__ void k_cdft_lr_init(int *lr, unsigned *nur, int S)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) {
        lr[2 * s] = INT_MAX;
        lr[2 * s + 1] = INT_MIN;
        nur[2 * s] = 0xffffffffu;
        nur[2 * s + 1] = 0u;
    }
}

// ---------------------------------------------------------------------------
// hist: count per (snapshot, lag) bucket. A CTA takes a 64 x 64 tile of grid
// nodes of one snapshot, held in registers (thread t: tile entries t + 256 k,
// so a warp reads 32 consecutive nodes of one grid row). Their lags span a
// few hundred values at most, so the counts are aggregated in shared memory
// first, one atomic per run of equal lags in a warp (global atomics only for
// tiles whose lag span exceeds kHistBins). Along a grid row the lag changes
// smoothly, so equal lags sit in consecutive lanes: a run is found with one
// shuffle and one ballot, where a general match of equal values costs far
// more when most lanes differ (a grid step moving the lag by a sample or more).
// ---------------------------------------------------------------------------
constexpr int kHistTile = 64;     // tile side (nodes)
constexpr int kHistBins = 2048;   // shared-memory buckets per CTA
constexpr int kTilePer = kHistTile * kHistTile / 256;  // tile entries per thread

// The tile's lags (INT_MIN outside the grid) and their range over the CTA
// (s_min > s_max when no node has a representable lag).
__device__ __forceinline__ void load_lag_tile(const CdftBatch &a, int s, int (&l)[kTilePer], int &s_min, int &s_max)
{
    const int tiles_j = (a.nlon + kHistTile - 1) / kHistTile;
    const int r0 = (blockIdx.x / tiles_j) * kHistTile, c0 = (blockIdx.x % tiles_j) * kHistTile;
    const int *Ls = a.candL + (size_t)s * a.G;
    if (threadIdx.x == 0) {
        s_min = INT_MAX;
        s_max = INT_MIN;
    }
    int lo = INT_MAX, hi = INT_MIN;
#pragma unroll
    for (int k = 0; k < kTilePer; ++k) {
        const int i = threadIdx.x + 256 * k;
        const int r = r0 + i / kHistTile, c = c0 + i % kHistTile;
        l[k] = (r < a.nrows && c < a.nlon) ? Ls[(int64_t)r * a.nlon + c] : INT_MIN;
        if (l[k] != INT_MIN) {
            lo = min(lo, l[k]);
            hi = max(hi, l[k]);
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, d));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, d));
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&s_min, lo);
        atomicMax(&s_max, hi);
    }
    __syncthreads();
}

// Runs of equal values over consecutive lanes: run_heads marks the lanes
// that start one (lane 0, or a value that differs from the previous lane's);
// run_len is the length of the run a head lane starts, run_head the head lane
// of this lane's run. Every lane of the warp takes part.
__device__ __forceinline__ unsigned run_heads(int v)
{
    const int lane = threadIdx.x & 31;
    const int prev = __shfl_up_sync(0xffffffffu, v, 1);
    return __ballot_sync(0xffffffffu, lane == 0 || prev != v);
}
__device__ __forceinline__ int run_len(unsigned heads, int lane)
{
    const unsigned above = heads & ~((2u << lane) - 1u);  // heads after this lane (none for lane 31)
    return (above ? __ffs(above) - 1 : 32) - lane;
}
__device__ __forceinline__ int run_head(unsigned heads, int lane)
{
    return 31 - __clz(heads & (0xffffffffu >> (31 - lane)));  // the last head at or before this lane
}

// Grid index of tile entry k of this thread.
__device__ __forceinline__ int64_t tile_node(const CdftBatch &a, int k)
{
    const int tiles_j = (a.nlon + kHistTile - 1) / kHistTile;
    const int i = threadIdx.x + 256 * k;
    return (int64_t)((blockIdx.x / tiles_j) * kHistTile + i / kHistTile) * a.nlon
         + (blockIdx.x % tiles_j) * kHistTile + i % kHistTile;
}

__global__ void __launch_bounds__(256) k_cdft_hist(CdftBatch a)
{
    __shared__ int s_cnt[kHistBins];
    __shared__ int s_min, s_max;
    const int s = blockIdx.y;
    const int lmin = a.lr[2 * s], bb = a.bbase[s], cap = a.bbase[s + 1] - bb;
    int l[kTilePer];
    load_lag_tile(a, s, l, s_min, s_max);
    if (s_max < s_min) return;  // no node with a representable lag (uniform)
    if (a.lr[2 * s + 1] - lmin >= cap) {  // more lags than the snapshot's bucket slots
        if (threadIdx.x == 0) atomicOr(a.err, ERR_LAG_RANGE);
        return;
    }
    const int tlo = s_min;
    const bool local = (int64_t)s_max - s_min < kHistBins;
    const int span = local ? s_max - s_min + 1 : 0;
    for (int i = threadIdx.x; i < span; i += blockDim.x) s_cnt[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < kTilePer; ++k) {
        const unsigned heads = run_heads(l[k]);
        if (((heads >> lane) & 1u) && l[k] != INT_MIN) {
            if (local)
                atomicAdd(s_cnt + (l[k] - tlo), run_len(heads, lane));
            else
                atomicAdd(a.count + bb + l[k] - lmin, run_len(heads, lane));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < span; i += blockDim.x)
        if (s_cnt[i]) atomicAdd(a.count + bb + tlo + i - lmin, s_cnt[i]);
}

// ---------------------------------------------------------------------------
// scan: one CTA (1024 threads) per snapshot.
// offs[b]  = offset of bucket b's candidates within the snapshot's order slice
// g2b      = the record of each combine group (bucket, snapshot, first
//            position in the order slice, size), groups of a bucket in a row
// nubase[s], delta[s] = the snapshot's bins (from its FDOA range).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_cdft_scan(CdftBatch a)
{
    __shared__ int s_c[1024], s_g[1024];
    const int s = blockIdx.x, t = threadIdx.x;
    const int b_first = a.bbase[s];
    const int lo_l = a.lr[2 * s], hi_l = a.lr[2 * s + 1];
    int NB = hi_l >= lo_l ? hi_l - lo_l + 1 : 0;
    if (NB > a.bbase[s + 1] - b_first) NB = 0;  // reported by k_cdft_hist
    const int per = (NB + 1023) / 1024;
    const int b0 = min(NB, t * per), b1 = min(NB, b0 + per);
    int c = 0, g = 0;
    for (int i = b0; i < b1; ++i) {
        const int n = a.count[b_first + i];
        c += n;
        g += (n + kCdftCombineGroup - 1) / kCdftCombineGroup;
    }
    s_c[t] = c;
    s_g[t] = g;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        const int vc = t >= d ? s_c[t - d] : 0, vg = t >= d ? s_g[t - d] : 0;
        __syncthreads();
        s_c[t] += vc;
        s_g[t] += vg;
        __syncthreads();
    }
    int oc = t ? s_c[t - 1] : 0, og = t ? s_g[t - 1] : 0;
    for (int i = b0; i < b1; ++i) {
        const int b = b_first + i;
        bool nd = a.count[b] > 0;
        if (a.delay != DG_DELAY_INTEGER)  // lags of the stencils of buckets i - 2 .. i + 1
            for (int d = -2; d <= 1 && !nd; ++d) nd = i + d >= 0 && i + d < NB && a.count[b + d] > 0;
        a.need[b] = nd ? 1 : 0;
        a.offs[b] = oc;
        const int n = a.count[b];
        const int ng = (n + kCdftCombineGroup - 1) / kCdftCombineGroup;
        for (int g = 0; g < ng; ++g)
            a.g2b[a.gbase[s] + og + g] =
                make_int4(b, s, oc + g * kCdftCombineGroup, min(kCdftCombineGroup, n - g * kCdftCombineGroup));
        oc += n;
        og += ng;
    }
    if (t == 0) {
        const float lo = unfkey(a.nur[2 * s]), hi = unfkey(a.nur[2 * s + 1]);
        // 64 bins: kCdftBinSpan steps over [lo, hi] (a little wider so that
        // rounding keeps every candidate inside) and kCdftBinPad more on each
        // side, so that every candidate's 6-point stencil is centred on it
        const float d = fmaxf((hi - lo) * (1.0f + 1e-5f) / (float)kCdftBinSpan, 1e-20f);
        a.nubase[s] = lo - (float)kCdftBinPad * d;
        a.delta[s] = d;
        if ((double)d * (double)a.M > kCdftMDelta) atomicOr(a.err, ERR_BIN_SPACING);
    }
}

// ---------------------------------------------------------------------------
// scatter: counting sort by lag bucket (the offsets come from the scan). A CTA
// takes the hist kernel's 64 x 64 tile of one snapshot. Its candidates are
// ranked per lag in shared memory (one atomic per run of equal lags in a
// warp, as in hist) and one global atomic per (tile, lag) reserves a
// contiguous range of the bucket: the candidates of one tile and lag sit
// together, which keeps the combine's surface writes close. The tile is
// then put in lag order in shared memory (local offsets from a prefix sum of
// the per-lag counts), so that consecutive threads write consecutive
// positions of each range: where a grid step moves the lag by a sample or
// more, nearly every lane of a warp has a lag of its own and writing in grid
// order would touch a cache line per lane. Tiles with longer runs of equal
// lags write in grid order (their writes are grouped already, and the
// reordering's barriers cost more than it gains), and so do tiles whose lag
// span exceeds kHistBins, with one global atomic per (warp, run).
// ---------------------------------------------------------------------------
constexpr int kTileN = kHistTile * kHistTile;

// Dynamic shared memory of k_cdft_scatter: per-lag counts (then local
// offsets) and range bases, then per lag-ordered position the packed
// (lag index, tile entry), the FDOA and, with LAGRANGE4, the fractional delay.
size_t scatter_smem_bytes(bool frac)
{
    return sizeof(int) * (2 * (size_t)kHistBins + (frac ? 3 : 2) * (size_t)kTileN);
}

// In-place exclusive prefix sum of v[0, n), n <= 8 * blockDim.x (256
// threads); returns the total. Every thread of the CTA calls it.
__device__ __forceinline__ int block_exclusive_scan(int *v, int n, int *s_warp)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int i0 = 8 * t;
    int x[8], sum = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        x[e] = i0 + e < n ? v[i0 + e] : 0;
        sum += x[e];
    }
    int inc = sum;  // inclusive scan of the threads' sums within the warp
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        const int ws = s_warp[w];
        if (w < warp) before += ws;
        total += ws;
    }
    int run = before + inc - sum;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        if (i0 + e < n) v[i0 + e] = run;
        run += x[e];
    }
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(256, 3) k_cdft_scatter(CdftBatch a)
{
    extern __shared__ __align__(16) int s_dyn[];
    int *s_cnt = s_dyn, *s_base = s_dyn + kHistBins;
    int *s_key = s_dyn + 2 * kHistBins;  // (lag index << 12) | tile entry
    float *s_nu = reinterpret_cast<float *>(s_key + kTileN);
    float *s_mu = s_nu + kTileN;  // LAGRANGE4 only
    __shared__ int s_min, s_max, s_warp[8], s_runs, s_valid;
    const int s = blockIdx.y;
    const int lmin = a.lr[2 * s], bb = a.bbase[s];
    if (a.lr[2 * s + 1] - lmin >= a.bbase[s + 1] - bb) return;  // reported by k_cdft_hist
    const bool frac = a.delay != DG_DELAY_INTEGER;
    int l[kTilePer];
    load_lag_tile(a, s, l, s_min, s_max);
    if (s_max < s_min) return;  // no node with a representable lag (uniform)
    const int tlo = s_min;
    const bool local = (int64_t)s_max - s_min < kHistBins;
    const int span = local ? s_max - s_min + 1 : 0;
    for (int i = threadIdx.x; i < span; i += blockDim.x) s_cnt[i] = 0;
    if (threadIdx.x == 0) s_runs = s_valid = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    int rank[kTilePer], runs = 0, valid = 0;
#pragma unroll
    for (int k = 0; k < kTilePer; ++k) {
        // one atomic per run of equal lags in the warp; the run's lanes take
        // consecutive ranks in lane order
        const unsigned heads = run_heads(l[k]);
        const int head = run_head(heads, lane);
        int base = 0;
        if (lane == head && l[k] != INT_MIN)
            base = local ? atomicAdd(s_cnt + (l[k] - tlo), run_len(heads, lane))
                         : atomicAdd(a.subcnt + bb + l[k] - lmin, run_len(heads, lane));
        rank[k] = __shfl_sync(0xffffffffu, base, head) + (lane - head);
        runs += __popc(heads);
        valid += __popc(__ballot_sync(0xffffffffu, l[k] != INT_MIN));
    }
    if (lane == 0) {
        atomicAdd(&s_runs, runs);
        atomicAdd(&s_valid, valid);
    }
    const size_t so = (size_t)s * a.G;
    __syncthreads();
    // lag order pays where runs are short (a mean under 4 lanes: measured,
    // it gains on a grid whose step moves the lag by 1-1.5 samples and loses
    // where the step moves it by 0.2); with longer runs the grid-order
    // writes are already grouped
    const bool lag_order = local && s_valid < 4 * s_runs;
    if (local) {
        // the global range of each (tile, lag)
        for (int i = threadIdx.x; i < span; i += blockDim.x) {
            const int n = s_cnt[i];
            s_base[i] = n ? atomicAdd(a.subcnt + bb + tlo + i - lmin, n) : 0;
        }
        if (!lag_order) __syncthreads();
    }
    if (!lag_order) {
        // grid order: every load before the first store (the stores may
        // alias the loads as far as the compiler knows)
        float nu[kTilePer];
#pragma unroll
        for (int k = 0; k < kTilePer; ++k) {
            if (l[k] == INT_MIN) continue;
            rank[k] += a.offs[bb + l[k] - lmin] + (local ? s_base[l[k] - tlo] : 0);
            nu[k] = a.candNu[so + tile_node(a, k)];
        }
#pragma unroll
        for (int k = 0; k < kTilePer; ++k) {
            if (l[k] == INT_MIN) continue;
            a.order[so + rank[k]] = (int)tile_node(a, k);
            a.nuS[so + rank[k]] = nu[k];
        }
        if (frac) {
#pragma unroll
            for (int k = 0; k < kTilePer; ++k)
                if (l[k] != INT_MIN) nu[k] = a.candMu[so + tile_node(a, k)];
#pragma unroll
            for (int k = 0; k < kTilePer; ++k)
                if (l[k] != INT_MIN) a.muS[so + rank[k]] = nu[k];
        }
        return;
    }
    // local offsets of the lags in the tile's lag order
    const int total = block_exclusive_scan(s_cnt, span, s_warp);
    // position p of lag index i goes to s_base[i] + p
    for (int i = threadIdx.x; i < span; i += blockDim.x)
        s_base[i] += a.offs[bb + tlo + i - lmin] - s_cnt[i];
    // lag order in shared memory (the FDOA loads stay coalesced, in grid order)
#pragma unroll
    for (int k = 0; k < kTilePer; ++k) {
        if (l[k] == INT_MIN) continue;
        const int li = l[k] - tlo, pos = s_cnt[li] + rank[k];
        const int64_t node = tile_node(a, k);
        s_key[pos] = (li << 12) | (int)(threadIdx.x + 256 * k);
        s_nu[pos] = a.candNu[so + node];
        if (frac) s_mu[pos] = a.candMu[so + node];
    }
    __syncthreads();
    const int tiles_j = (a.nlon + kHistTile - 1) / kHistTile;
    const int64_t r0 = (int64_t)(blockIdx.x / tiles_j) * kHistTile, c0 = (int64_t)(blockIdx.x % tiles_j) * kHistTile;
    for (int p = threadIdx.x; p < total; p += blockDim.x) {
        const int key = s_key[p], e = key & (kTileN - 1);
        const int64_t dst = so + s_base[key >> 12] + p;
        a.order[dst] = (int)((r0 + e / kHistTile) * a.nlon + c0 + e % kHistTile);
        a.nuS[dst] = s_nu[p];
        if (frac) a.muS[dst] = s_mu[p];
    }
}

// ---------------------------------------------------------------------------
// contract (FP32 CUDA cores): CTA = (bucket, 64 chunks); thread = 4 bins x 4
// chunks. Per sample m of the chunk: z_L[bM + m] for the CTA's 64 chunks and
// V[m][q] (the snapshot's table) in shared memory, 16 complex MACs per thread.
// ---------------------------------------------------------------------------
constexpr int kCtChunks = 64;  // chunks per CTA
constexpr int kCtSub = 32;     // samples per shared-memory pass

__global__ void __launch_bounds__(256) k_cdft_vtable(float2 *V, const float *nubase, const float *delta, int M, int S)
{
    const int s = blockIdx.y;
    const float b0 = nubase[s], d = delta[s];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M * 64; i += gridDim.x * blockDim.x) {
        const int m = i >> 6, q = i & 63;
        float sn, cs;  // bin frequency in FP32 as the combine forms it; exact product split
        sincospif(2.0f * frac_mul(fmaf((float)q, d, b0), (float)m), &sn, &cs);
        V[(size_t)s * M * 64 + i] = make_float2(cs, sn);
    }
}

template <int FMT>
__global__ void __launch_bounds__(256) k_cdft_contract_f32(CdftBatch a)
{
    __shared__ __align__(16) float2 zs[kCtSub][kCtChunks + 1];  // +1: staging stores 2-way, not 32-way
    __shared__ __align__(16) float2 vs[kCtSub][64];
    const int b = blockIdx.x;
    if (!a.need[b]) return;
    const int s = step_of(a.bbase, a.S, b);
    const StepDesc sd = a.sd[s];
    const int N = sd.n, M = a.M;
    const int B = (N + M - 1) / M;
    const int c0 = blockIdx.y * kCtChunks;
    if (c0 >= B) return;
    const int L = a.lr[2 * s] + (b - a.bbase[s]);
    const float2 *V = a.V + (size_t)s * M * 64;
    const int tq = threadIdx.x & 15, tc = threadIdx.x >> 4;  // bins 4tq..4tq+3, chunks 4tc..4tc+3
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int m0 = 0; m0 < M; m0 += kCtSub) {
        __syncthreads();
        // z' for 32 samples x 64 chunks; the modulation phase is per sample
        for (int i = threadIdx.x; i < kCtSub * kCtChunks; i += 256) {
            const int mm = i & (kCtSub - 1), cc = i / kCtSub;
            const int n = (c0 + cc) * M + m0 + mm, n2 = n + L;
            float2 z = make_float2(0.f, 0.f);
            if (c0 + cc < B && n < N && n2 >= 0 && n2 < N) {
                const float2 x = IQ<FMT>::load(sd.y1, n), y = IQ<FMT>::load(sd.y2, n2);
                z.x = fmaf(x.x, y.x, x.y * y.y);
                z.y = fmaf(x.y, y.x, -x.x * y.y);
            }
            zs[mm][cc] = z;
        }
        for (int i = threadIdx.x; i < kCtSub * 64; i += 256) vs[i >> 6][i & 63] = V[(size_t)(m0 + (i >> 6)) * 64 + (i & 63)];
        __syncthreads();
#pragma unroll 4
        for (int mm = 0; mm < kCtSub; ++mm) {
            const float2 z0 = zs[mm][4 * tc], z1 = zs[mm][4 * tc + 1], z2 = zs[mm][4 * tc + 2], z3 = zs[mm][4 * tc + 3];
            // vs rows are 512 B and 4 tq is even: these 16-byte loads are aligned
            const float4 v01 = *reinterpret_cast<const float4 *>(&vs[mm][4 * tq]);
            const float4 v23 = *reinterpret_cast<const float4 *>(&vs[mm][4 * tq + 2]);
            const float zr[4] = {z0.x, z1.x, z2.x, z3.x}, zi[4] = {z0.y, z1.y, z2.y, z3.y};
            const float vr[4] = {v01.x, v01.z, v23.x, v23.z}, vi[4] = {v01.y, v01.w, v23.y, v23.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fmaf(zr[i], vr[j], fmaf(-zi[i], vi[j], acc[i][j].x));
                    acc[i][j].y = fmaf(zr[i], vi[j], fmaf(zi[i], vr[j], acc[i][j].y));
                }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int ch = c0 + 4 * tc + i;
        if (ch < B) {  // planar row: 64 real parts, then 64 imaginary parts
            float *w = a.W + ((size_t)b * a.Bmax + ch) * 128 + 4 * tq;
            *reinterpret_cast<float4 *>(w) = make_float4(acc[i][0].x, acc[i][1].x, acc[i][2].x, acc[i][3].x);
            *reinterpret_cast<float4 *>(w + 64) = make_float4(acc[i][0].y, acc[i][1].y, acc[i][2].y, acc[i][3].y);
        }
    }
}

// ---------------------------------------------------------------------------
// superchunk: merge the per-chunk DFTs of a bucket into super-chunks of
// Mc = R M samples, exactly at the bin frequencies:
//     U_c(nu_q) = sum_{r<R} e^{j 2 pi nu_q r M} W_{cR + r}(nu_q).
// The combine then interpolates U_c between bins, and its error is governed
// by Mc Delta instead of M Delta; k_cdft_tiles picks Mc so that Mc Delta
// stays within the same bound. One thread per (bucket, bin); each reads its own
// bin of chunks cR .. cR + R - 1 and writes super-chunk c in place (c <= cR,
// and later super-chunks read only later chunks).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_cdft_superchunk(CdftBatch a, int NBT)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)NBT * 64) return;
    const int bg = (int)(t >> 6), q = (int)(t & 63);
    if (!a.need[bg]) return;  // no candidate's stencil reaches it: W rows were not written
    const int s = step_of(a.bbase, a.S, bg);
    const int M = a.M, R = a.Mcs[s] / a.M;
    if (R == 1) return;
    const int B = (a.sd[s].n + M - 1) / M;
    const float nq = a.nubase[s] + (float)q * a.delta[s];
    float ex, ey;  // e^{j 2 pi nu_q M}
    sincospif(2.0f * frac_mul(nq, (float)M), &ey, &ex);
    float *Wb = a.W + (size_t)bg * a.Bmax * 128;
    for (int c = 0; c * R < B; ++c) {
        float ux = 0.f, uy = 0.f;
        const int r1 = min(R, B - c * R);
        // blocks of 16 chunks: the rotation is anchored at each block's first
        // chunk and stepped within it; the block's loads are issued together
        for (int r0 = 0; r0 < r1; r0 += 16) {
            float px = 1.f, py = 0.f;
            if (r0 > 0) sincospif(2.0f * frac_mul(nq, (float)(r0 * M)), &py, &px);
            const float *w = Wb + (size_t)(c * R + r0) * 128;
            float wx[16], wy[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                wx[r] = r0 + r < r1 ? w[(size_t)r * 128 + q] : 0.f;
                wy[r] = r0 + r < r1 ? w[(size_t)r * 128 + 64 + q] : 0.f;
            }
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                if (r0 + r >= r1) break;
                ux = fmaf(px, wx[r], fmaf(-py, wy[r], ux));
                uy = fmaf(px, wy[r], fmaf(py, wx[r], uy));
                const float nx = fmaf(px, ex, -py * ey);
                py = fmaf(px, ey, py * ex);
                px = nx;
            }
        }
        Wb[(size_t)c * 128 + q] = ux;
        Wb[(size_t)c * 128 + 64 + q] = uy;
    }
}

// ---------------------------------------------------------------------------
// combine: kCdftCombineGroup candidates of one bucket per CTA,
// kCdftCombinePer per thread; the bucket's super-chunk
// DFTs stream through shared memory in segments of kSeg. Each candidate
// interpolates the DFT of every super-chunk at its own FDOA from the six
// bins around it (Lagrange, the FDOA between the third and fourth),
// rotates it by the super-chunk's phase e^{j 2 pi nu c Mc}, and sums.
// With the Lagrange4 fractional delay the candidate's correlation is, by
// linearity, sum_{m=-1..2} w_m(mu) C_{L+m}(nu) with the 4-tap weights of its
// fractional delay mu: the same sum over the buckets of lags L - 1 .. L + 2,
// each weighted.
// ---------------------------------------------------------------------------
constexpr int kSeg = 32;

template <typename T, bool FRAC>
__global__ void __launch_bounds__(kCdftCombineThreads) k_cdft_combine(CdftBatch a, T *surf)
{
    // per (super-)chunk and bin: the DFT value (re, im)
    __shared__ __align__(16) float2 ws[kSeg][64];
    // one CTA per combine group of the batch's upper bound; groups past a
    // snapshot's last are -1 in the scan's group map. Every thread reads the
    // group's record and its snapshot's constants itself (broadcast loads),
    // so the bucket's DFTs and the candidates are one round trip behind it.
    const int4 gr = a.g2b[blockIdx.x];
    const int b = gr.x;
    if (b < 0) return;  // uniform
    const int s = gr.y, n = gr.w;
    const int M = a.Mcs[s];
    const int B = (a.sd[s].n + M - 1) / M;
    const float nbase = a.nubase[s], inv = 1.0f / a.delta[s];
    constexpr bool frac = FRAC;  // a.delay != DG_DELAY_INTEGER
    constexpr int mlo = frac ? -1 : 0, mhi = frac ? 2 : 0;  // lag offsets of the stencil
    // the first segment of DFTs depends on the bucket only: its loads travel
    // together with the candidates' below
    {
        const float *Wb = a.W + (size_t)(b + mlo) * a.Bmax * 128;
        for (int i = threadIdx.x; i < min(kSeg, B) * 64; i += kCdftCombineThreads) {
            const int ch = i >> 6, q = i & 63;
            const float *row = Wb + (size_t)ch * 128;
            ws[ch][q] = make_float2(row[q], row[64 + q]);
        }
    }
    const size_t sp0 = (size_t)s * a.G + gr.z;
    int c[kCdftCombinePer], q0[kCdftCombinePer];
    float w[kCdftCombinePer][6], lw[kCdftCombinePer][4], ex[kCdftCombinePer], ey[kCdftCombinePer],
        px[kCdftCombinePer], py[kCdftCombinePer], cx[kCdftCombinePer], cy[kCdftCombinePer], nu[kCdftCombinePer];
#pragma unroll
    for (int k = 0; k < kCdftCombinePer; ++k) {
        const int j = threadIdx.x + k * kCdftCombineThreads;
        const bool act = j < n;
        c[k] = act ? a.order[sp0 + j] : -1;
        nu[k] = act ? a.nuS[sp0 + j] : nbase + (float)kCdftBinPad * a.delta[s];
        // 6-point Lagrange interpolation on bins q0 - 2 .. q0 + 3 with q0 the
        // bin at or below the FDOA, kept in [2, 60] (the padding keeps the
        // FDOA in [q0, q0 + 1]); t = offset from bin q0
        const float u = (nu[k] - nbase) * inv;
        q0[k] = max(kCdftBinPad, min(62 - kCdftBinPad, __float2int_rd(u)));
        const float t = u - (float)q0[k];
        const float a2 = t + 2.f, a1 = t + 1.f, b1 = t - 1.f, b2 = t - 2.f, b3 = t - 3.f;
        const float t01 = t * b1, t23 = b2 * b3, s21 = a2 * a1;
        w[k][0] = -(a1 * t01 * t23) * (1.f / 120.f);
        w[k][1] = (a2 * t01 * t23) * (1.f / 24.f);
        w[k][2] = -(s21 * b1 * t23) * (1.f / 12.f);
        w[k][3] = (s21 * t * t23) * (1.f / 12.f);
        w[k][4] = -(s21 * t01 * b3) * (1.f / 24.f);
        w[k][5] = (s21 * t01 * b2) * (1.f / 120.f);
        // the 4-tap weights of the fractional delay mu (lags L - 1 .. L + 2)
        const float mu = (frac && act) ? a.muS[sp0 + j] : 0.f;
        lw[k][0] = frac ? -mu * (mu - 1.f) * (mu - 2.f) * (1.f / 6.f) : 1.f;
        lw[k][1] = (mu + 1.f) * (mu - 1.f) * (mu - 2.f) * 0.5f;
        lw[k][2] = -(mu + 1.f) * mu * (mu - 2.f) * 0.5f;
        lw[k][3] = (mu + 1.f) * mu * (mu - 1.f) * (1.f / 6.f);
        // chunk-to-chunk phase step e^{j 2 pi nu M}
        sincospif(2.0f * frac_mul(nu[k], (float)M), &ey[k], &ex[k]);
        cx[k] = cy[k] = 0.f;
    }
    for (int m = mlo; m <= mhi; ++m) {
        const float *Wb = a.W + (size_t)(b + m) * a.Bmax * 128;
        float wm[kCdftCombinePer][6];  // bin weights times the lag's weight
#pragma unroll
        for (int k = 0; k < kCdftCombinePer; ++k)
#pragma unroll
            for (int e = 0; e < 6; ++e) wm[k][e] = w[k][e] * lw[k][m - mlo];
        for (int s0 = 0; s0 < B; s0 += kSeg) {
            const int slen = min(kSeg, B - s0);
            if (s0 > 0 || m > mlo) {
                __syncthreads();
                for (int i = threadIdx.x; i < slen * 64; i += kCdftCombineThreads) {
                    const int ch = i >> 6, q = i & 63;
                    const float *row = Wb + (size_t)(s0 + ch) * 128;
                    ws[ch][q] = make_float2(row[q], row[64 + q]);
                }
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kCdftCombinePer; ++k) {
                // phase of the segment's first sample, e^{j 2 pi nu s0 M}
                if (s0 == 0) {
                    px[k] = 1.f;
                    py[k] = 0.f;
                } else {
                    sincospif(2.0f * frac_mul(nu[k], (float)s0 * (float)M), &py[k], &px[k]);
                }
#pragma unroll 4
                for (int i = 0; i < slen; ++i) {
                    const float2 *wr = &ws[i][q0[k] - 2];
                    float zx = 0.f, zy = 0.f;
#pragma unroll
                    for (int e = 0; e < 6; ++e) {
                        const float2 v = wr[e];
                        zx = fmaf(wm[k][e], v.x, zx);
                        zy = fmaf(wm[k][e], v.y, zy);
                    }
                    cx[k] = fmaf(px[k], zx, fmaf(-py[k], zy, cx[k]));
                    cy[k] = fmaf(px[k], zy, fmaf(py[k], zx, cy[k]));
                    const float nx = fmaf(px[k], ex[k], -py[k] * ey[k]);
                    py[k] = fmaf(px[k], ey[k], py[k] * ex[k]);
                    px[k] = nx;
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kCdftCombinePer; ++k)
        if (c[k] >= 0) {
            const float pw = fmaf(cx[k], cx[k], cy[k] * cy[k]);
            surf[(size_t)(a.k0 + s) * a.G + c[k]] = (T)(a.acc == DG_ACC_POWER ? pw : sqrtf(pw));
        }
}

// ---------------------------------------------------------------------------
// tiles: one warp, after the scan. Per snapshot of the batch: its lag
// buckets (from the lag range), the tensor-core tile layout (128 lags x one
// chunk unless padding the lags to blocks of 128 more than doubles the tile
// count, or a chunk above kLagTileMaxChunk is not a multiple of it), the tile offsets, and the
// combine chunk: the longest power-of-two multiple of M with
// Mc x bin spacing <= kCdftMDelta, up to the first length that covers the
// snapshot and at most 2^24. Also the work counters.
// ---------------------------------------------------------------------------
__global__ void k_cdft_tiles(CdftBatch a)
{
    // one warp; lane l plans snapshots l, l + 32, ...; the tile offsets are a
    // warp prefix sum
    const int lane = threadIdx.x;
    if (blockIdx.x != 0 || lane >= 32) return;
    int running = 0, hrunning = 0;
    unsigned long long rows = 0, cands = 0;
    for (int s0 = 0; s0 < a.S; s0 += 32) {
        const int s = s0 + lane;
        int tiles = 0, htiles = 0;
        if (s < a.S) {
            const int lo = a.lr[2 * s], hi = a.lr[2 * s + 1];
            int NB = hi >= lo ? hi - lo + 1 : 0;
            if (NB > a.bbase[s + 1] - a.bbase[s]) NB = 0;
            const int n = a.sd[s].n, M = a.M;
            const int B = (n + M - 1) / M;
            const int t_row = (int)(((int64_t)NB * B + 127) / 128), t_lag = B * ((NB + 127) / 128);
            const int t_hk = B * ((NB + kHkLags - 1) / kHkLags);
            const int NFB = NB / 128, rem = NB - 128 * NFB;
            const int t_mix = NFB * B + (int)(((int64_t)rem * B + 127) / 128);
            // 0: row tiles, 1: lag tiles, 2: Hankel tiles
            // AUTO: lag tiles unless padding the lags to whole blocks of 128
            // more than doubles the tile count; and when the last block holds
            // fewer than 64 lags, those lags go into row tiles (packed (lag,
            // chunk) rows, about two lag tiles' cost each) instead of a mostly
            // empty block (3: mixed). Hankel tiles only on request (measured
            // slower: their per-phase MMAs of N = 64 re-read the 128-row operand
            // eight times per K step)
            // lag tiles stage their chunk in windows of kLagTileMaxChunk
            // samples: chunks up to that length, or whole multiples of it
            int lay = 0;
            const bool windows = M <= kLagTileMaxChunk || M % kLagTileMaxChunk == 0;
            if (a.mma && a.tiles_mode == DG_TILES_HANKEL && M <= kLagTileMaxChunk) lay = 2;
            else if (a.mma && windows && a.tiles_mode == DG_TILES_LAGS) lay = 1;
            else if (a.mma && windows && a.tiles_mode == DG_TILES_AUTO && t_lag <= 2 * t_row)
                lay = (NFB >= 1 && rem > 0 && rem < 64) ? 3 : 1;
            a.layout[s] = lay;
            tiles = lay == 2 ? 0 : lay == 3 ? t_mix : lay ? t_lag : t_row;
            htiles = lay == 2 ? t_hk : 0;
            int64_t Mc = M;
            const double d = (double)a.delta[s];
            while (Mc < n && 2 * Mc <= ((int64_t)1 << 24) && (double)(2 * Mc) * d <= kCdftMDelta) Mc *= 2;
            a.Mcs[s] = (int)Mc;
            rows += (unsigned long long)NB * B;
            cands += (unsigned long long)a.G * ((n + Mc - 1) / Mc);
        }
        int incl = tiles, hincl = htiles;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d);
            const int hy = __shfl_up_sync(0xffffffffu, hincl, d);
            if (lane >= d) {
                incl += y;
                hincl += hy;
            }
        }
        if (s < a.S) {
            a.tbase[s] = running + incl - tiles;
            a.hbase[s] = hrunning + hincl - htiles;
        }
        running += __shfl_sync(0xffffffffu, incl, 31);
        hrunning += __shfl_sync(0xffffffffu, hincl, 31);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        rows += __shfl_xor_sync(0xffffffffu, rows, d);
        cands += __shfl_xor_sync(0xffffffffu, cands, d);
    }
    if (lane == 0) {
        a.tbase[a.S] = running;
        a.hbase[a.S] = hrunning;
        if (a.work) {
            a.work[0] += rows;
            a.work[1] += cands;
        }
    }
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
static unsigned grid_for(int64_t n, int per, int cap = 152 * 16)
{
    int64_t b = (n + per - 1) / per;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

__global__ void __launch_bounds__(256) k_ecef_split(const double *__restrict__ xyz, int64_t G, float *__restrict__ xf)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < G; p += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const dfl v = df_from(xyz[c * G + p]);
            xf[(2 * c) * G + p] = v.hi;
            xf[(2 * c + 1) * G + p] = v.lo;
        }
    }
}

cudaError_t launch_ecef_split(const double *xyz, int64_t G, float *xyzf, cudaStream_t st)
{
    k_ecef_split<<<grid_for(G, 256), 256, 0, st>>>(xyz, G, xyzf);
    return cudaGetLastError();
}

cudaError_t launch_cdft_geo(const CdftBatch &a, cudaStream_t st)
{
    k_cdft_lr_init<<<(a.S + 127) / 128, 128, 0, st>>>(a.lr, a.nur, a.S);
    dim3 grid(grid_for(a.G, 256 * 4, 152 * 8), (unsigned)a.S);
    k_cdft_geo<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cdft_plan(const CdftBatch &a, int NBT, cudaStream_t st)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(a.count, 0, sizeof(int) * (size_t)NBT, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.subcnt, 0, sizeof(int) * (size_t)NBT, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.need, 0, sizeof(int) * (size_t)NBT, st)) != cudaSuccess) return e;
    const int64_t tiles = (int64_t)((a.nrows + kHistTile - 1) / kHistTile) * ((a.nlon + kHistTile - 1) / kHistTile);
    dim3 gh((unsigned)tiles, (unsigned)a.S);
    k_cdft_hist<<<gh, 256, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_cdft_scan<<<a.S, 1024, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
        const size_t sm = scatter_smem_bytes(a.delay != DG_DELAY_INTEGER);
        if ((e = cudaFuncSetAttribute(k_cdft_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
            cudaSuccess)
            return e;
        k_cdft_scatter<<<gh, 256, sm, st>>>(a);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (a.mma) return cudaSuccess;  // the FP32 table serves the CUDA-core contraction only
    dim3 gv(grid_for((int64_t)a.M * 64, 256, 64), (unsigned)a.S);
    k_cdft_vtable<<<gv, 256, 0, st>>>(a.V, a.nubase, a.delta, a.M, a.S);
    return cudaGetLastError();
}

cudaError_t launch_cdft_contract_fp32(const CdftBatch &a, int NBT, int fmt, cudaStream_t st)
{
    dim3 grid((unsigned)NBT, (unsigned)((a.Bmax + kCtChunks - 1) / kCtChunks));
    switch (fmt) {
    case DG_IQ_C64: k_cdft_contract_f32<DG_IQ_C64><<<grid, 256, 0, st>>>(a); break;
    case DG_IQ_CI16: k_cdft_contract_f32<DG_IQ_CI16><<<grid, 256, 0, st>>>(a); break;
    default: k_cdft_contract_f32<DG_IQ_CI8><<<grid, 256, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_cdft_superchunk(const CdftBatch &a, int NBT, cudaStream_t st)
{
    const int64_t n = (int64_t)NBT * 64;
    k_cdft_superchunk<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, NBT);
    return cudaGetLastError();
}

cudaError_t launch_cdft_combine(const CdftBatch &a, float *surf, cudaStream_t st)
{
    if (a.delay == DG_DELAY_INTEGER)
        k_cdft_combine<float, false><<<(unsigned)a.ngroups, kCdftCombineThreads, 0, st>>>(a, surf);
    else
        k_cdft_combine<float, true><<<(unsigned)a.ngroups, kCdftCombineThreads, 0, st>>>(a, surf);
    return cudaGetLastError();
}

cudaError_t launch_cdft_tiles(const CdftBatch &a, cudaStream_t st)
{
    k_cdft_tiles<<<1, 32, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace dg
