// dg_noalloc.cu -- the cost surface computed without allocating device memory.
//
// Some callers may not allocate GPU memory while they process data: a
// real-time receiver chain that reserves all of its device memory once at
// start-up so that no allocation can stall or fail in the middle of a pass,
// or a host program whose device memory is owned by another allocator (a
// framework's caching allocator, a pool with a fixed quota) that must not be
// bypassed. dg_create allocates (grid ECEF, captures, per-snapshot surfaces),
// so those callers use dg_cost_surface_noalloc instead: it runs the same
// kernels with all of its scratch in one statically sized device array that
// belongs to the library.
//
// The array below is reserved on every GPU on which this library's device
// code is loaded, and stays reserved until the process exits. Its device
// address is looked up once per device (with that device current) through
// cudaGetSymbolAddress: in host code the name g_noalloc_scratch is only a
// host-side stand-in and must never be passed to a kernel.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "dg_internal.cuh"

namespace dg {
namespace {

constexpr size_t kNoAllocScratchBytes = DG_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_addr_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

__global__ void k_noalloc_steps(StepDesc *steps, const char *y1, const char *y2, int K, int n, int fmt,
                                size_t step_bytes)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < K) {
        steps[k].y1 = y1 + step_bytes * (size_t)k;
        steps[k].y2 = y2 + step_bytes * (size_t)k;
        steps[k].n = n;
        steps[k].fmt = fmt;
    }
}

thread_local char g_msg[384];

dg_status nfail(dg_status st, const char *msg)
{
    std::snprintf(g_msg, sizeof g_msg, "%s", msg);
    return st;
}

dg_status ncuda(cudaError_t e, const char *what)
{
    std::snprintf(g_msg, sizeof g_msg, "%s: %s", what, cudaGetErrorString(e));
    return DG_ECUDA;
}

bool finite_eph(const dg_ephem &e)
{
    const double *v = &e.p1[0];
    for (int t = 0; t < 12; ++t)
        if (!std::isfinite(v[t])) return false;
    return true;
}

}  // namespace
}  // namespace dg

using namespace dg;

extern "C" const char *dg_noalloc_last_error(void) { return g_msg; }

extern "C" dg_status dg_cost_surface_noalloc(const dg_grid *grid, const dg_ephem *eph, int32_t K,
                                             double fs_hz, double fc_hz, int32_t fmt, const void *y1,
                                             const void *y2, int64_t n_samples, const dg_options *opt,
                                             void *out, void *cuda_stream)
{
    g_msg[0] = 0;
    // ---- argument checks (same rules as dg_create / dg_load_capture) ----------
    if (!grid || !eph || !y1 || !y2 || !out) return nfail(DG_EINVAL, "a pointer argument is NULL");
    if (!(std::isfinite(grid->lat0_deg) && std::fabs(grid->lat0_deg) < 89.0) || !std::isfinite(grid->lon0_deg))
        return nfail(DG_EINVAL, "grid centre must be finite, latitude within +-89 deg");
    if (!(grid->dlat_m > 0 && grid->dlon_m > 0 && std::isfinite(grid->dlat_m) && std::isfinite(grid->dlon_m)))
        return nfail(DG_EINVAL, "grid spacing must be positive and finite");
    if (grid->nlat < 1 || grid->nlon < 1) return nfail(DG_EINVAL, "nlat and nlon must be >= 1");
    if (K < 1 || K > 65535) return nfail(DG_EINVAL, "K must be in [1, 65535]");
    if (!(fs_hz > 0 && std::isfinite(fs_hz)) || !(fc_hz > 0 && std::isfinite(fc_hz)))
        return nfail(DG_EINVAL, "fs_hz and fc_hz must be positive and finite");
    size_t bps = fmt == DG_IQ_C64 ? 8 : fmt == DG_IQ_CI16 ? 4 : fmt == DG_IQ_CI8 ? 2 : 0;
    if (!bps) return nfail(DG_EINVAL, "unknown IQ format");
    if (n_samples < 1 || n_samples > ((int64_t)1 << 30)) return nfail(DG_EINVAL, "n_samples must be in [1, 2^30]");
    dg_options o;
    dg_options_default(&o);
    if (opt) o = *opt;
    if ((o.delay != DG_DELAY_INTEGER && o.delay != DG_DELAY_LAGRANGE4) ||
        (o.acc != DG_ACC_POWER && o.acc != DG_ACC_MAG) || (o.prec != DG_PREC_FP32 && o.prec != DG_PREC_FP64) ||
        o.algo != DG_ALGO_DIRECT)
        return nfail(DG_EINVAL, "unknown delay, accumulation, precision or algorithm option");
    if (o.row0 < 0 || o.row0 >= grid->nlat || o.nrows < 0 || o.row0 + o.nrows > grid->nlat)
        return nfail(DG_EINVAL, "row shard outside the grid");
    if (!direct_rows_ok(o.prec, o.rows))
        return nfail(DG_EINVAL, "rows must be 0, 4, 8 or 16 (FP32) or 0, 2 or 4 (FP64)");
    for (int k = 0; k < K; ++k)
        if (!finite_eph(eph[k])) return nfail(DG_EINVAL, "an ephemeris is not finite");

    // ---- scratch layout: [ecef 3G doubles | surfaces K G | steps K | eph K*12 | err] ----
    const int nrows = o.nrows ? o.nrows : grid->nlat - o.row0;
    const int64_t G = (int64_t)nrows * grid->nlon;
    const size_t esz = o.prec == DG_PREC_FP64 ? 8 : 4;
    const size_t b_xyz = up256(sizeof(double) * 3 * (size_t)G);
    const size_t b_surf = up256(esz * (size_t)G * (size_t)K);
    const size_t b_steps = up256(sizeof(StepDesc) * (size_t)K);
    const size_t b_eph = up256(sizeof(double) * 12 * (size_t)K);
    const size_t need = b_xyz + b_surf + b_steps + b_eph + 256;
    if (need > kNoAllocScratchBytes) {
        std::snprintf(g_msg, sizeof g_msg,
                      "this call needs %zu bytes of scratch (24*G + %zu*K*G + 128*K + alignment, "
                      "G = %lld nodes, K = %d); the static scratch holds %zu bytes",
                      need, esz, (long long)G, K, kNoAllocScratchBytes);
        return DG_EINVAL;
    }
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return ncuda(e, "cudaGetSymbolAddress(scratch)");
    char *p = static_cast<char *>(base);
    double *xyz = reinterpret_cast<double *>(p);
    void *surf = p + b_xyz;
    StepDesc *steps = reinterpret_cast<StepDesc *>(p + b_xyz + b_surf);
    double *eph_d = reinterpret_cast<double *>(p + b_xyz + b_surf + b_steps);
    unsigned *err = reinterpret_cast<unsigned *>(p + b_xyz + b_surf + b_steps + b_eph);
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // The array keeps the previous call's contents: clear the error word; every
    // other region is fully rewritten below before it is read.
    if ((e = cudaMemsetAsync(err, 0, sizeof(unsigned), s)) != cudaSuccess) return ncuda(e, "cudaMemsetAsync");
    // pageable source: the copy has been staged when this returns
    if ((e = cudaMemcpyAsync(eph_d, eph, sizeof(double) * 12 * (size_t)K, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return ncuda(e, "cudaMemcpyAsync(ephemerides)");
    GridDev gd;
    gd.lat0_rad = grid->lat0_deg * (kPi / 180.0);
    gd.lon0_rad = grid->lon0_deg * (kPi / 180.0);
    gd.dlat_m = grid->dlat_m;
    gd.dlon_m = grid->dlon_m;
    gd.nlat = grid->nlat;
    gd.nlon = grid->nlon;
    gd.row0 = o.row0;
    gd.nrows = nrows;
    if ((e = launch_grid_ecef(gd, xyz, s)) != cudaSuccess) return ncuda(e, "grid kernel");
    k_noalloc_steps<<<(K + 127) / 128, 128, 0, s>>>(steps, static_cast<const char *>(y1),
                                                    static_cast<const char *>(y2), K, (int)n_samples, fmt,
                                                    bps * (size_t)n_samples);
    if ((e = cudaGetLastError()) != cudaSuccess) return ncuda(e, "step-table kernel");
    CorrArgs a{};
    a.xyz = xyz;
    a.eph = eph_d;
    a.steps = steps;
    a.surf = surf;
    a.err = err;
    a.nrows = nrows;
    a.nlon = grid->nlon;
    a.G = G;
    a.fs = fs_hz;
    a.lambda = kC / fc_hz;
    a.K = K;
    a.fmt = fmt;
    a.delay = o.delay;
    a.acc = o.acc;
    a.prec = o.prec;
    a.rows = o.rows;
    if ((e = launch_corr_direct(a, s)) != cudaSuccess) return ncuda(e, "correlation kernel");
    if ((e = launch_accumulate(surf, K, G, o.prec, out, s)) != cudaSuccess) return ncuda(e, "accumulation kernel");
    unsigned herr = 0;
    if ((e = cudaMemcpyAsync(&herr, err, sizeof herr, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return ncuda(e, "cudaMemcpyAsync(error word)");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return ncuda(e, "cudaStreamSynchronize");
    if (herr & ERR_NU_RANGE)
        return nfail(DG_EUNSUPPORTED, "a candidate's FDOA exceeds 0.2 fs; the correlation kernels do not handle it");
    if (herr) return nfail(DG_EUNSUPPORTED, "a candidate's lag |D| exceeds 1e9 samples");
    return DG_OK;
}
