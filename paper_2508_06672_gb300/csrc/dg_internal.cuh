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
enum : unsigned { ERR_NU_RANGE = 1u, ERR_LAG_RANGE = 2u };

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
cudaError_t launch_grid_ecef(const GridDev &g, double *xyz, cudaStream_t s);

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
};

// Launch the direct correlation for all K snapshots (one launch).
cudaError_t launch_corr_direct(const CorrArgs &a, cudaStream_t s);

// out[p] = sum_k surf[k][p], k in order.
cudaError_t launch_accumulate(const void *surf, int K, int64_t G, int prec, void *out,
                              cudaStream_t s);

// ---------------------------------------------------------------------------
// Chunked-DFT evaluation (DG_ALGO_CDFT), csrc/dg_cdft.cu.
// ---------------------------------------------------------------------------
// Lag range of every snapshot: lr[2k] = min L, lr[2k+1] = max L.
cudaError_t launch_cdft_range(const double *xyz, const double *eph, int K, int64_t G, double fs, double lambda,
                              int *lr, unsigned *err, cudaStream_t s);

struct CdftStepArgs {
    const double *xyz;            // [3][G]
    const double *eph_k;          // [12] of this snapshot
    const StepDesc *sd_k;         // this snapshot's captures (device)
    const int *lr_k;              // {min L, max L} of this snapshot (device)
    int64_t G;
    double fs, lambda;
    int NB;                       // buckets = max L - min L + 1 (host copy)
    int M, B;                     // samples per chunk, chunks
    int fmt, acc, contract;
    int *candB;                   // [G] bucket of each candidate
    double *candNu;               // [G] nu of each candidate
    int *order;                   // [G] candidates sorted by bucket
    int *count, *cursor;          // [NB]
    unsigned long long *nulo, *nuhi;  // [NB] ordered keys of the FDOA range
    int *offs, *gofs;             // [NB + 1]
    double *nulo_d;               // [NB]
    double *delta;                // [1] bin spacing
    float2 *W;                    // [NB][B][64]
    void *surf_k;                 // this snapshot's slice of the surfaces (float)
};

// memsets + histogram + scan + scatter of one snapshot
cudaError_t launch_cdft_plan(const CdftStepArgs &a, cudaStream_t s);
// W[bucket][chunk][bin] of one snapshot
cudaError_t launch_cdft_contract(const CdftStepArgs &a, cudaStream_t s);
// per-candidate sums over chunks into the snapshot's surface slice
cudaError_t launch_cdft_combine(const CdftStepArgs &a, cudaStream_t s);

// Argmax record written by launch_argmax.
struct ArgmaxResult {
    double val;
    int64_t idx;                 // -1 if every value is NaN
    double lat_rad, lon_rad;     // node of idx in the grid g (if idx >= 0)
};

// Argmax of v[0..n) (ties to the lowest index, NaN never wins); tmp must hold
// argmax_tmp_bytes(n) bytes; writes *res (device).
size_t argmax_tmp_bytes(int64_t n);
cudaError_t launch_argmax(const void *v, int64_t n, int prec, const GridDev &g, void *tmp,
                          ArgmaxResult *res, int *launches, cudaStream_t s);

}  // namespace dg
