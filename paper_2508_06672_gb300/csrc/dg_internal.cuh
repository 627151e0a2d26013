// dg_internal.cuh -- device helpers and launcher declarations shared by the
// translation units of libdg. Not part of the public ABI (include/dg.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dg.h"

namespace dg {

constexpr double kC = 299792458.0;               // speed of light, m/s
constexpr double kA = 6378137.0;                 // WGS-84 semi-major axis, m
constexpr double kF = 1.0 / 298.257223563;       // WGS-84 flattening
constexpr double kPi = 3.14159265358979323846;

constexpr int kThreads = 256;                    // threads per correlation CTA
constexpr int kWarps = kThreads / 32;

// Error bits latched by kernels into the context's device error word.
enum : unsigned { ERR_NU_RANGE = 1u, ERR_LAG_RANGE = 2u, ERR_BIN_SPACING = 4u, ERR_TIMEOUT = 8u };

// A grid (or a shard of rows of it) as the kernels see it.
struct GridDev {
    double lat0_rad, lon0_rad;   // centre node
    double dlat_m, dlon_m;       // spacing in metres at the centre latitude
    int nlat, nlon;              // whole grid
    int row0, nrows;             // shard rows [row0, row0 + nrows)
};

// One snapshot's captures in device memory.
struct StepDesc {
    const void *y1;
    const void *y2;
    int n;                       // samples per receiver
    int fmt;                     // DG_IQ_*
};

// ---------------------------------------------------------------------------
// Geometry (Sec. III, Eq. 3-10), FP64. Every operation is an explicitly
// rounded IEEE operation (no FMA contraction), in a fixed order, so that the
// integer lag round(D) / floor(D) is reproducible on any IEEE machine that
// evaluates the same expression in the same order.
// e = [p1 v1 p2 v2] (ECEF), lambda = c / fc.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void geometry(double cx, double cy, double cz, const double *e,
                                         double fs, double lambda, double &D, double &nu)
{
    // Eq. 3: r_i = p_i - p_c
    const double r1x = __dsub_rn(e[0], cx), r1y = __dsub_rn(e[1], cy), r1z = __dsub_rn(e[2], cz);
    const double r2x = __dsub_rn(e[6], cx), r2y = __dsub_rn(e[7], cy), r2z = __dsub_rn(e[8], cz);
    // Eq. 4: rho_i = |r_i|
    const double rho1 = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(r1x, r1x), __dmul_rn(r1y, r1y)),
                                             __dmul_rn(r1z, r1z)));
    const double rho2 = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(r2x, r2x), __dmul_rn(r2y, r2y)),
                                             __dmul_rn(r2z, r2z)));
    // Eq. 5-6: f_i = -(r_i . v_i) / (rho_i lambda)
    const double f1 = -__ddiv_rn(__dadd_rn(__dadd_rn(__dmul_rn(r1x, e[3]), __dmul_rn(r1y, e[4])),
                                           __dmul_rn(r1z, e[5])),
                                 __dmul_rn(rho1, lambda));
    const double f2 = -__ddiv_rn(__dadd_rn(__dadd_rn(__dmul_rn(r2x, e[9]), __dmul_rn(r2y, e[10])),
                                           __dmul_rn(r2z, e[11])),
                                 __dmul_rn(rho2, lambda));
    // Eq. 7-9: dtau = tau_2 - tau_1, D = dtau * fs (samples); Eq. 8, 10: nu = (f_2 - f_1) / fs
    const double dtau = __ddiv_rn(__dsub_rn(rho2, rho1), kC);
    D = __dmul_rn(dtau, fs);
    nu = __ddiv_rn(__dsub_rn(f2, f1), fs);
}

// ---------------------------------------------------------------------------
// Double-float arithmetic: a value is hi + lo with two floats (about 46
// significant bits), built from error-free transformations (two-sum, FMA
// products). It runs on the FP32 pipes, which on this chip are far wider than
// FP64. Used for the per-(candidate, snapshot) geometry of the chunked-DFT
// path; the integer lag is still decided by the FP64 expression wherever the
// double-float value lies near a rounding boundary.
// ---------------------------------------------------------------------------
struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl df_from(double d)
{
    const float h = (float)d;
    return {h, (float)(d - (double)h)};
}
__device__ __forceinline__ dfl df_fast_two_sum(float a, float b)
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ dfl df_two_sum(float a, float b)
{
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    dfl s = df_two_sum(a.hi, b.hi);
    const dfl t = df_two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = df_fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return df_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, {-b.hi, -b.lo}); }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
// a + b without the renormalisation of the low words' sum: relative error
// ~2^-44 of |a| + |b| (enough here: see geometry_df).
__device__ __forceinline__ dfl df_add_fast(dfl a, dfl b)
{
    const dfl s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ dfl df_sub_fast(dfl a, dfl b) { return df_add_fast(a, {-b.hi, -b.lo}); }
// sqrt of a double-float: one Newton correction of the FP32 root. The
// residual a.hi - y^2 of y = sqrtf(a.hi) is exact in FP32, so one FMA gives it.
__device__ __forceinline__ dfl df_sqrt(dfl a)
{
    const float y = sqrtf(a.hi);
    const float r = fmaf(-y, y, a.hi) + a.lo;
    return df_fast_two_sum(y, __fdividef(r, 2.f * y));
}

// a / b for a double-float quotient: the FP32 quotient plus one correction
// from the exact-by-FMA residual (relative error ~1e-14).
__device__ __forceinline__ dfl df_div_fast(dfl a, dfl b)
{
    const float q1 = __fdividef(a.hi, b.hi);
    const float r = fmaf(-q1, b.hi, a.hi) + (a.lo - q1 * b.lo);
    return df_fast_two_sum(q1, __fdividef(r, b.hi));
}

// Eq. 3-10 for the chunked-DFT plan. The lag needs D = (rho2 - rho1) fs / c
// to ~1e-7 samples (so that Eq. 9 rounds it as the FP64 expression does
// wherever D is farther than 1e-6 from a rounding boundary), i.e. the ranges
// to ~1e-6 m out of 1e6 m: double-float. The candidate and the receivers
// are double-float splits of the FP64 values: a pair of floats keeps 48 of
// the 53 significand bits, a relative error of at most 2^-48 (~3e-8 m on
// ECEF coordinates of 7e6 m, against the 1e-6 sample = 1.5e-5 m at 20 MHz
// that round_df leaves as its margin). Every sum carries an error of at
// most ~2^-44 of its operands' magnitude (~1e-6 m on the range vectors,
// ~1e-7 m on the ranges), and fs / c is a double-float constant.
// The FDOA, nu = (f2 - f1) / fs with f_i = -(r_i . v_i) / (rho_i lambda),
// is a difference of two range rates of ~7 km/s whose result is used as the
// phase rate over the whole capture; at nodes where |C| is a small remainder
// of a cancelling sum, an error of 1e-9 cycles per sample already shows at
// 1e-4 in |C|^2. So the range rates r_i . v_i / rho_i and their difference
// are double-float too, and nu is rounded to FP32 once, at the end.
__device__ __forceinline__ void geometry_df(dfl x, dfl y, dfl z, const dfl *e, dfl fs_over_c, dfl inv_lam_fs,
                                            dfl &D, float &nu)
{
    const dfl r1x = df_sub_fast(e[0], x), r1y = df_sub_fast(e[1], y), r1z = df_sub_fast(e[2], z);
    const dfl r2x = df_sub_fast(e[6], x), r2y = df_sub_fast(e[7], y), r2z = df_sub_fast(e[8], z);
    const dfl rho1 = df_sqrt(df_add_fast(df_add_fast(df_mul(r1x, r1x), df_mul(r1y, r1y)), df_mul(r1z, r1z)));
    const dfl rho2 = df_sqrt(df_add_fast(df_add_fast(df_mul(r2x, r2x), df_mul(r2y, r2y)), df_mul(r2z, r2z)));
    D = df_mul(df_sub_fast(rho2, rho1), fs_over_c);
    const dfl q1 = df_div_fast(df_add_fast(df_add_fast(df_mul(r1x, e[3]), df_mul(r1y, e[4])), df_mul(r1z, e[5])), rho1);
    const dfl q2 = df_div_fast(df_add_fast(df_add_fast(df_mul(r2x, e[9]), df_mul(r2y, e[10])), df_mul(r2z, e[11])), rho2);
    const dfl n = df_mul(df_sub_fast(q1, q2), inv_lam_fs);  // (f2 - f1) lambda / (lambda fs)
    nu = n.hi + n.lo;
}

// frac(nu * x) for an integer-valued x < 2^24, to ~1e-7 cycles: the product
// is split exactly into p + e with an FMA, and p - floor(p) is exact.
__device__ __forceinline__ float frac_mul(float nu, float x)
{
    const float p = nu * x;
    const float e = fmaf(nu, x, -p);
    return (p - floorf(p)) + e;
}

// Eq. 9 on a double-float D: round half away from zero, in FP32 only.
// Returns false (undecided) when |D| >= 2^22 or when D lies within 1e-6 of a
// rounding boundary; the caller then decides with the FP64 expression.
__device__ __forceinline__ bool round_df(dfl D, int &L)
{
    const float ah = fabsf(D.hi);
    if (!(ah < 4194304.0f)) return false;
    const float al = D.hi < 0.f ? -D.lo : D.lo;  // |D| = ah + al
    float n = floorf(ah);
    float f = (ah - n) + al;                     // ah - n is exact
    if (f < 0.f) {
        n -= 1.f;
        f += 1.f;
    } else if (f >= 1.f) {
        n += 1.f;
        f -= 1.f;
    }
    if (fabsf(f - 0.5f) < 1e-6f || f < 1e-6f || f > 1.f - 1e-6f) return false;
    const int mag = (int)n + (f > 0.5f ? 1 : 0);
    L = D.hi < 0.f ? -mag : mag;
    return true;
}

// floor(D) of a double-float D and the remainder mu = D - floor(D) in
// [0, 1), in FP32 only; false when |D| >= 2^22 (the caller then uses FP64).
// (Lagrange4 is continuous across integer D, so a lag off by one next to an
// integer gives the same interpolated sample; no rounding margin is needed.)
__device__ __forceinline__ bool floor_df(dfl D, int &L, float &mu)
{
    if (!(fabsf(D.hi) < 4194304.0f)) return false;
    float n = floorf(D.hi);
    float f = (D.hi - n) + D.lo;  // D.hi - n is exact
    if (f < 0.f) {
        n -= 1.f;
        f += 1.f;
    } else if (f >= 1.f) {
        n += 1.f;
        f -= 1.f;
    }
    L = (int)n;
    mu = fminf(fmaxf(f, 0.f), 1.f);
    return true;
}

// Integer lag of the delay mode: Eq. 9 (round half away from zero) or floor.
__device__ __forceinline__ int lag_of(double D, int delay_mode)
{
    return delay_mode == DG_DELAY_INTEGER ? (int)round(D) : (int)floor(D);
}

// Node (i, j) of a grid -> geodetic latitude/longitude in radians, with the
// angular spacing metres / (meridian radius) and metres / (parallel radius).
struct GridStep {
    double dlat, dlon;
};

__device__ __forceinline__ GridStep grid_step(const GridDev &g)
{
    const double e2 = kF * (2.0 - kF);
    const double s = sin(g.lat0_rad);
    const double w = __dsqrt_rn(__dsub_rn(1.0, __dmul_rn(__dmul_rn(e2, s), s)));
    const double m = __ddiv_rn(kA * (1.0 - e2), __dmul_rn(__dmul_rn(w, w), w));
    const double n = __ddiv_rn(kA, w);
    GridStep st;
    st.dlat = __ddiv_rn(g.dlat_m, m);
    st.dlon = __ddiv_rn(g.dlon_m, __dmul_rn(n, cos(g.lat0_rad)));
    return st;
}

__device__ __forceinline__ void grid_node(const GridDev &g, const GridStep &st, int i, int j,
                                          double &lat, double &lon)
{
    lat = __dadd_rn(g.lat0_rad, __dmul_rn(__dsub_rn((double)i, 0.5 * (double)(g.nlat - 1)), st.dlat));
    lon = __dadd_rn(g.lon0_rad, __dmul_rn(__dsub_rn((double)j, 0.5 * (double)(g.nlon - 1)), st.dlon));
}

// ---------------------------------------------------------------------------
// IQ loaders: sample idx of an interleaved I,Q array as (re, im), exact.
// ---------------------------------------------------------------------------
template <int FMT> struct IQ;
template <> struct IQ<DG_IQ_C64> {
    static __device__ __forceinline__ float2 load(const void *b, int idx)
    {
        return __ldg(reinterpret_cast<const float2 *>(b) + idx);
    }
};
template <> struct IQ<DG_IQ_CI16> {
    static __device__ __forceinline__ float2 load(const void *b, int idx)
    {
        const short2 v = __ldg(reinterpret_cast<const short2 *>(b) + idx);
        return make_float2((float)v.x, (float)v.y);
    }
};
template <> struct IQ<DG_IQ_CI8> {
    static __device__ __forceinline__ float2 load(const void *b, int idx)
    {
        const char2 v = __ldg(reinterpret_cast<const char2 *>(b) + idx);
        return make_float2((float)v.x, (float)v.y);
    }
};

// ---------------------------------------------------------------------------
// Launchers (host functions; each returns the launch's cudaError_t).
// ---------------------------------------------------------------------------
struct ArgmaxResult;
// centre (device, optional): take the grid's centre from an argmax record, as
// the refinement grid does (its latitude / longitude rounded through degrees
// exactly as the host would pass them)
cudaError_t launch_grid_ecef(const GridDev &g, double *xyz, cudaStream_t s, const ArgmaxResult *centre = nullptr);

cudaError_t launch_step_geometry(const GridDev &g, const double *xyz, const double *eph_k,
                                 double fs, double lambda, int delay_mode, int *lag, double *D,
                                 double *nu, cudaStream_t s);

struct CorrArgs {
    const double *xyz;           // [3][G] shard ECEF
    const double *eph;           // [K][12]
    const StepDesc *steps;       // [K] device table
    void *surf;                  // [K][G] per-snapshot |C|^2 or |C| (float or double)
    unsigned *err;               // device error word
    int nrows, nlon;
    int64_t G;
    double fs, lambda;
    int K;
    int fmt;                     // common format of all steps
    int delay, acc, prec;
    int rows;                    // grid rows per thread (dg_options.rows; 0 = default)
};

// Admissible dg_options.rows of the direct kernel for a precision.
inline bool direct_rows_ok(int prec, int rows)
{
    return rows == 0 || (prec == DG_PREC_FP64 ? (rows == 2 || rows == 4) : (rows == 4 || rows == 8 || rows == 16));
}

// Launch the direct correlation for all K snapshots (one launch).
cudaError_t launch_corr_direct(const CorrArgs &a, cudaStream_t s);

// out[p] = sum_k surf[k][p], k in order.
cudaError_t launch_accumulate(const void *surf, int K, int64_t G, int prec, void *out,
                              cudaStream_t s);

// ---------------------------------------------------------------------------
// Chunked-DFT evaluation (DG_ALGO_CDFT), csrc/dg_cdft.cu, csrc/dg_cdft_mma.cu.
// A batch is S consecutive snapshots [k0, k0 + S) processed by the same
// launches. Global bucket ids of snapshot s are bbase[s] .. bbase[s+1]-1, one
// per lag lr[2s] .. lr[2s+1]; combine groups of snapshot s are gbase[s] ..
// gbase[s+1]-1 (an upper bound; surplus CTAs exit).
// ---------------------------------------------------------------------------
constexpr int kCdftCombineThreads = 128;
// candidates per combine thread. Threads x candidates per CTA, combine ms per
// step on the large workload (4001^2, K = 50, 8 super-chunks per candidate) /
// on mid: 128 x 3: 12.03 / 0.237; 128 x 2: 12.62 / 0.239; 128 x 4: 12.28 /
// 0.241; 64 x 8: 13.12 / 0.253 (earlier, on mid: 256 x 4 and 512 x 2 slower)
constexpr int kCdftCombinePer = 3;
constexpr int kCdftCombineGroup = kCdftCombineThreads * kCdftCombinePer;  // candidates per combine CTA

struct CdftBatch {
    const double *xyz;            // [3][G]
    const double *eph;            // [S][12] (first snapshot of the batch)
    const StepDesc *sd;           // [S] captures
    int S, k0;
    int64_t G;
    int nrows, nlon;              // shard shape (G = nrows * nlon)
    double fs, lambda;
    int M, Bmax, acc;
    unsigned *err;
    int *lr;                      // [S][2] lag range
    unsigned *nur;                // [S][2] FDOA range (ordered float keys)
    const int *bbase, *gbase;     // [S + 1] (device)
    const float *xyzf;            // [6][G] ECEF as double-float: x hi, x lo, y hi, y lo, z hi, z lo
    const float *ephf;            // [S][24] ephemerides as double-float (hi, lo) pairs
    float fsc_hi, fsc_lo;         // fs / c as double-float (samples per metre)
    float ilf_hi, ilf_lo;         // 1 / (lambda fs) as double-float
    int *candL;                   // [S][G] lag (INT_MIN: not representable)
    float *candNu;                // [S][G] FDOA / fs
    int *order;                   // [S][G] candidates sorted by (bucket, bin)
    float *nuS;                   // [S][G] their FDOAs, in the same order
    int4 *g2b;                    // [groups] per combine group: x bucket (-1: none), y snapshot, z its first
                                  // position in the snapshot's order slice, w its candidates
    int *count;                   // [NBT]
    int *offs;                    // [NBT]
    int *subcnt;                  // [NBT] fill cursor of each bucket (scatter)
    float *nubase, *delta;        // [S] bins nu_q = nubase + q delta
    float2 *V;                    // [S][M][64] DFT table e^{j 2 pi nu_q m}
    float *W;                     // [NBT][Bmax][128]: per chunk 64 bins, re[64] | im[64]
    int *tbase;                   // [S + 1] first tensor-core tile of each snapshot (k_cdft_tiles)
    int *hbase;                   // [S + 1] first Hankel tile of each snapshot (k_cdft_tiles)
    int *layout;                  // [S] 1: tiles of 128 lags x one chunk, 0: 128 (lag, chunk) rows
    int *Mcs;                     // [S] combine chunk: a power-of-two multiple of M (k_cdft_tiles)
    unsigned long long *work;     // [2] lag x chunk rows, candidate x super-chunk pairs (or NULL)
    int tiles_mode;               // DG_TILES_*; tensor-core contraction or not (mma)
    int mma;
    int ngroups;                  // combine groups of the batch (upper bound; unused ones are -1 in g2b)
    const void *btab;             // [S][M/32][2][128 x 32] 16-bit DFT operand (tensor cores)
    float zscale;                 // lag products are multiplied by this before 16-bit rounding
    unsigned wait_polls;          // poll limit of the tensor-core pipeline's waits; 0 = the default
    int delay;                    // DG_DELAY_INTEGER: lag round(D); DG_DELAY_LAGRANGE4: lag floor(D) and
                                  // the candidate combines the lags L - 1 .. L + 2 (fractional delay)
    float *candMu;                // [S][G] fractional delay mu = D - floor(D) (Lagrange4 only)
    float *muS;                   // [S][G] mu in sorted order (Lagrange4 only)
    int *need;                    // [NBT] 1: the bucket's per-lag DFT rows are computed (scan)
};

// Bucket b's rows are needed when a candidate's lag stencil reaches it: its
// own candidates (integer lags), or those of buckets b - 2 .. b + 1
// (Lagrange4 combines lags L - 1 .. L + 2).

// Status of the network-layer calls (dg_nn_*): the message of the last
// failure on this thread (dg_nn_last_error).
dg_status nn_fail(dg_status st, const char *fmt, ...);
dg_status nn_done(cudaError_t e, const char *what);

// What the tensor-core contraction needs of one job: one snapshot batch of
// one context (its plan done: tile bases, lag ranges, layouts, the
// need flags, the DFT operand tables). Several jobs can share one persistent
// launch; their tiles are numbered job after job.
struct TcJob {
    const StepDesc *sd;           // [S] captures
    const int *tbase, *bbase, *lr, *layout, *need;
    float *W;                     // per-lag DFT rows
    const void *btab;             // DFT operand tables, [S][M/32] stages
    unsigned *err;                // the context's latched error word
    int S, M, Bmax;
    float zscale;
};
TcJob tc_job(const CdftBatch &a, const void *btab);
// job_tiles[0..n]: prefix sum of the jobs' tile counts (one thread, device)
cudaError_t launch_tc_job_tiles(const TcJob *jobs, int n, int *job_tiles, cudaStream_t s);
// one persistent launch over every tile of n jobs (device array), all of
// the same capture format and contraction arithmetic
cudaError_t launch_cdft_contract_jobs(const TcJob *jobs, int n, const int *job_tiles, int grid, int fmt, int mode,
                                      unsigned wait_polls, cudaStream_t s);

cudaError_t launch_cdft_geo(const CdftBatch &a, cudaStream_t s);
// xyzf[6][G] = double-float split of xyz[3][G]
cudaError_t launch_ecef_split(const double *xyz, int64_t G, float *xyzf, cudaStream_t s);
cudaError_t launch_cdft_plan(const CdftBatch &a, int NBT, cudaStream_t s);
cudaError_t launch_cdft_contract_fp32(const CdftBatch &a, int NBT, int fmt, cudaStream_t s);
cudaError_t launch_cdft_combine(const CdftBatch &a, float *surf, cudaStream_t s);
// per snapshot: lag buckets, tile layout, tiles (tbase), combine chunk, work
// (one warp)
cudaError_t launch_cdft_tiles(const CdftBatch &a, cudaStream_t s);
// W[bucket][c] <- sum over the Mc / M chunks b of super-chunk c of
// e^{j 2 pi nu_q (b M - c Mc)} W[bucket][b] (in place; Mc > M)
cudaError_t launch_cdft_superchunk(const CdftBatch &a, int NBT, cudaStream_t s);
// tensor-core contraction (dg_cdft_mma.cu): mode DG_CONTRACT_BF16 / FP16 /
// BF16X3 / FP16X3; a persistent launch of `grid` CTAs over the batch's tiles
cudaError_t launch_cdft_btab(const CdftBatch &a, int mode, void *btab, cudaStream_t s);
cudaError_t launch_cdft_contract_mma(const CdftBatch &a, int grid, int fmt, int mode, cudaStream_t s);
// The Hankel tiles of the batch (k_cdft_contract_hk), persistent over `grid` CTAs.
cudaError_t launch_cdft_contract_hankel(const CdftBatch &a, int grid, int fmt, int mode, cudaStream_t s);
size_t cdft_btab_bytes(int mode, int M);  // per snapshot
// Lag tiles (128 consecutive lags of one chunk share one y1 segment and one
// y2 window, staged once in shared memory) need chunk <= this.
constexpr int kLagTileMaxChunk = 1024;
constexpr int kHkLags = 512;                     // lags of one Hankel tile (8 phases of 64)
// Snapshots per batch on the tensor-core path (the contraction caches their
// tables in shared memory).
constexpr int kTcMaxSnapshots = 64;

// CDFT chunk bounds: the longest chunk; the longest the automatic choice
// takes (longer chunks shorten the combine but lengthen the tables and the
// contraction's operand stream: 1024 was fastest on the 1001^2 and 4001^2
// workloads); and the bound on (samples summed per DFT) x (bin spacing), in
// cycles, for the 6-point Lagrange interpolation of the combine. The bins
// are padded by two on each side of the snapshot's FDOA range, so every
// candidate lies between the third and fourth nodes of its stencil
// (t in [0, 1]); there the error of interpolating a DFT of length L is at
// most |prod_{k=-2..3} (t - k)| / 6! (2 pi L Delta)^6 <= 4.9e-3 (2 pi L Delta)^6
// of the coherent sum, 4.7e-6 at this bound. The plan rejects a chunk above
// it; the automatic chunk and the super-chunks keep below it.
constexpr int kCdftMaxChunk = 16384;
constexpr int kCdftAutoMaxChunk = 1024;
// The tensor-core path takes automatic chunks up to kCdftAutoMaxChunkTc while
// a batch keeps kCdftMinTilesPerSm lag tiles per SM (the host's estimate).
// The cap is set by accuracy: the tensor cores' FP32 accumulation adds a
// relative error that grows with the number of MMAs summed into one
// accumulator (measured on the 4001^2 footprint against FP64, split fp16
// products: 1.2e-5 at 1024-sample chunks, 1.5e-4 at 16384, at the peak), so
// chunks are kept to 2048 samples (about 2.5e-5) and longer sums are formed
// in FP32 on the CUDA cores (super-chunks).
constexpr int kCdftAutoMaxChunkTc = 2048;
constexpr int kCdftMinTilesPerSm = 16;
// Automatic chunk cap of a refinement surface: its few lags per snapshot give
// few (lag, chunk) rows, and shorter chunks turn the same tensor work into
// more and shorter tiles, spread over more SMs.
constexpr int kCdftRefineMaxChunk = 256;
constexpr double kCdftMDelta = 5.0e-2;
constexpr int kCdftBinPad = 2;                  // bins outside the FDOA range on each side
constexpr int kCdftBinSpan = 63 - 2 * kCdftBinPad;  // bin steps across the FDOA range

// Threshold detection (dg_detect.cu). cap: power of two <= kDetectCap candidates
// (the sort keeps value + index of each in static shared memory, 32 KiB).
constexpr int kDetectCap = 2048;
struct DetectPeak {
    int64_t index;
    int i, j;
    double lat_rad, lon_rad, value;
};
cudaError_t launch_detect(const void *v, int prec, const GridDev &g, double thr, int r, int cap, int max_peaks,
                          int *count, int64_t *cand, DetectPeak *out, cudaStream_t s);

// Argmax record written by launch_argmax.
struct ArgmaxResult {
    double val;
    int64_t idx;                 // -1 if every value is NaN
    double lat_rad, lon_rad;     // node of idx in the grid g (if idx >= 0)
    double sub_lat_rad, sub_lon_rad;  // parabolic three-point estimate around it
};

// Argmax of v[0..n) (ties to the lowest index, NaN never wins); tmp must hold
// argmax_tmp_bytes(n) bytes; writes *res (device).
size_t argmax_tmp_bytes(int64_t n);
// The refinement grid centred on an argmax record (device): the same
// degrees round trip as the host's dg_grid of the local grid.
__device__ __forceinline__ void centre_on(GridDev &g, const ArgmaxResult *c)
{
    g.lat0_rad = (c->lat_rad * (180.0 / kPi)) * (kPi / 180.0);
    g.lon0_rad = (c->lon_rad * (180.0 / kPi)) * (kPi / 180.0);
}

// The fix of a step from its argmax records (device), as dg_argmax_refine
// assembles it on the host; fine may be NULL (no refinement, n = 0).
cudaError_t launch_make_fix(const ArgmaxResult *coarse, const ArgmaxResult *fine, const GridDev &g, int n,
                            dg_fix *out, cudaStream_t s);

cudaError_t launch_argmax(const void *v, int64_t n, int prec, const GridDev &g, void *tmp,
                          ArgmaxResult *res, int *launches, cudaStream_t s, const ArgmaxResult *centre = nullptr);

// ---------------------------------------------------------------------------
// Coarse delay-Doppler maps back-projected onto the grid's cells (the input
// of the learned proposal), csrc/dg_coarse.cu.
// ---------------------------------------------------------------------------
struct CoarseStep {
    int l0, nlag;                 // lags l0 .. l0 + nlag - 1 (node lags, Eq. 9)
    double nu_lo, delta, nu_c;    // bins nu_lo + q delta; chunk turning frequency
    double mu;                    // mean of the map
};

struct CoarseArgs {
    const double *xyz;            // [3][G] node ECEF (whole grid)
    int64_t G;
    int nlat, nlon;
    const float *xyzf;            // [6][G] node ECEF as double-float (x hi, x lo, y hi, ...)
    const double *eph;            // [K][12]
    const float *ephf;            // [K][24] ephemerides as double-float
    const StepDesc *steps;        // [K]
    int K;
    double fs, lambda;
    float fsc_hi, fsc_lo;         // fs / c as double-float
    float ilf_hi, ilf_lo;         // 1 / (lambda fs) as double-float
    int Q, M, nlag_cap, nb_max;   // bins, chunk, lag and chunk capacities
    int *lag;                     // [K][G] node lags
    float *nu;                    // [K][G] node FDOAs
    int *lmm;                     // [K][2] lag min / max
    unsigned long long *nmm;      // [K][2] FDOA min / max (ordered keys)
    CoarseStep *st;               // [K]
    float2 *P;                    // [K][nb_max][nlag_cap] chunk sums
    float *A;                     // [K][nlag_cap][Q] the maps |X|^2
    double *part;                 // [K][ceil(nlag_cap / 32)] partial sums of A
    float *maps;                  // [K][nlat - 1][nlon - 1]
    unsigned *err;
};
int coarse_bin_tiles(int nlag_cap);
// The whole coarse pipeline (7 launches; *launches += 7).
cudaError_t launch_coarse(const CoarseArgs &a, cudaStream_t s, int *launches);

}  // namespace dg
