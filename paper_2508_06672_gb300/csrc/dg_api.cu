// dg_api.cu -- host implementation of the C ABI declared in include/dg.h.
//
// The context owns every device buffer of the hot path: shard ECEF [3][G],
// ephemerides [K][12], per-snapshot captures (raw format, not widened), the
// per-snapshot surfaces [K][G] (scratch for the ordered accumulation), the
// argmax scratch and the refinement buffers. All allocation is
// stream-ordered (cudaMallocAsync / cudaFreeAsync) on the context's stream.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "dg_internal.cuh"

using namespace dg;

namespace {

thread_local std::string g_thread_error;

struct Step {
    int fmt = -1;
    int64_t n = 0;
    void *y1 = nullptr, *y2 = nullptr;
    size_t cap = 0;  // bytes per receiver buffer
    bool loaded = false;
};

struct TimedLaunch {
    int cls;
    cudaEvent_t a, b;
};

struct CdftLayout {  // batches and bucket / group bases of one grid size
    struct Batch {
        int k0, S, base;      // snapshots k0 .. k0 + S - 1; offset of its bases
        int64_t nbt, groups;  // lag slots and combine groups (upper bounds)
    };
    int64_t G = -1;
    double diam = 0.0;      // grid diameter bound the lag slots were sized for
    std::vector<Batch> batches;
    int s_max = 0;
    int64_t nbt_max = 0, groups_max = 0;
    int *bbase = nullptr, *gbase = nullptr;  // device, per batch: [S + 1] each
};

struct CdftRun {  // one chunked-DFT surface, phase by phase (run_surface_cdft)
    GridDev gd{};
    const double *xyz = nullptr;
    int64_t G = 0;
    void *surf = nullptr, *out = nullptr;
    bool refine = false, mma = false;
    CdftLayout *L = nullptr;
    std::vector<int> Ms;  // chunk of each batch of snapshots
};

struct CdftBufs {  // chunked-DFT scratch, grown on demand
    int *lr = nullptr;
    CdftLayout main_layout, loc_layout;
    std::vector<double> main_span;  // FDOA span estimates per snapshot (main grid)
    std::vector<double> main_lags;  // and lag-count estimates
    CdftRun main_run;               // the main surface's last run (its batches' arguments)
    int *layout = nullptr, *Mcs = nullptr;
    unsigned long long *work = nullptr;
    unsigned *nur = nullptr;
    float *nubase = nullptr;
    size_t s_cap = 0;
    int *candL = nullptr, *order = nullptr;
    float *candNu = nullptr, *nuS = nullptr;
    float *candMu = nullptr, *muS = nullptr;  // Lagrange4: fractional delays
    size_t mu_cap = 0;
    int *need = nullptr;
    size_t sg_cap = 0;
    int4 *g2b = nullptr;
    size_t g2b_cap = 0;
    float *xyzf = nullptr;
    size_t xyzf_cap = 0;
    float *ephf = nullptr;
    size_t ephf_cap = 0;
    int *count = nullptr, *offs = nullptr, *subcnt = nullptr;
    size_t nb_cap = 0;
    float *delta = nullptr;
    float2 *V = nullptr;
    size_t v_cap = 0;
    float *W = nullptr;
    size_t w_cap = 0;
    int *tbase = nullptr, *hbase = nullptr;
    void *btab = nullptr;
    size_t btab_cap = 0;
};

struct LocalGrid {  // refinement buffers, grown on demand
    double *xyz = nullptr;
    void *surf = nullptr;
    void *cost = nullptr;
    size_t g_cap = 0;
};

struct CoarseBufs {  // coarse delay-Doppler maps (dg_coarse_maps), grown on demand
    int *lag = nullptr;
    float *nu = nullptr;
    int *lmm = nullptr;
    unsigned long long *nmm = nullptr;
    CoarseStep *st = nullptr;
    float2 *P = nullptr;
    float *A = nullptr;
    double *part = nullptr;
    size_t lag_cap = 0, nu_cap = 0, lmm_cap = 0, nmm_cap = 0, st_cap = 0, P_cap = 0, A_cap = 0, part_cap = 0;
    int Q = 0, M = 0, nlag_cap = 0, nb_max = 0;  // shape of the last maps (Q = 0: none yet)
};

}  // namespace

struct dg_ctx {
    dg_grid grid{};
    dg_options opt{};
    int K = 0;
    double fs = 0, fc = 0, lambda = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    int sm_count = 1;
    GridDev gd{};
    int64_t G = 0;
    int64_t xyz_cap = 0;                // nodes the ECEF buffer holds
    ArgmaxResult *reg_res = nullptr;    // dg_search_regions: argmax per region (device)
    ArgmaxResult *reg_host = nullptr;   // pinned mirror
    size_t reg_cap = 0;
    double *xyz = nullptr;
    double *eph = nullptr;
    std::vector<dg_ephem> eph_host;
    std::vector<Step> steps;
    StepDesc *steps_d = nullptr;
    std::vector<StepDesc> steps_h;
    bool steps_dirty = true;
    void *surf = nullptr;
    size_t surf_bytes = 0;
    void *amax_tmp = nullptr;
    size_t amax_tmp_bytes = 0;
    ArgmaxResult *amax_res = nullptr;
    ArgmaxResult *amax_host = nullptr;  // pinned
    int *det_count = nullptr;
    int64_t *det_cand = nullptr;
    DetectPeak *det_out = nullptr;
    unsigned *err_d = nullptr;
    unsigned *err_h = nullptr;          // pinned mirror
    LocalGrid loc;
    CdftBufs cd;
    CoarseBufs co;
    int cd_chunk_min = 0, cd_chunk_max = 0;              // chunks it used
    // whole-step CUDA graph (dg_graph_*)
    ArgmaxResult *amax_fine = nullptr;  // refinement argmax (device)
    dg_fix *fix_dev = nullptr;
    dg_fix *fix_host = nullptr;         // pinned
    cudaGraphExec_t graph = nullptr;
    int64_t graph_launches = 0;         // kernels per replay
    uint64_t steps_gen = 1, graph_gen = 0;  // capture buffers / formats / lengths generation
    std::string err;
    int64_t launches = 0;
    std::vector<TimedLaunch> pending;
    double ms[DG_K_NCLASS] = {};
    int64_t nl[DG_K_NCLASS] = {};
};

namespace {

dg_status fail(dg_ctx *c, dg_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_thread_error = buf;
    return st;
}

#define CK(ctx, call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? DG_ENOMEM : DG_ECUDA, "%s: %s", \
                        #call, cudaGetErrorString(e_));                                        \
    } while (0)

size_t iq_bytes(int fmt)
{
    switch (fmt) {
    case DG_IQ_C64: return 8;
    case DG_IQ_CI16: return 4;
    case DG_IQ_CI8: return 2;
    default: return 0;
    }
}

bool finite3(const double *v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

// Record kernel timing events around a launch when timing is on.
struct Timed {
    dg_ctx *c;
    int cls;
    cudaEvent_t a = nullptr, b = nullptr;
    Timed(dg_ctx *c_, int cls_) : c(c_), cls(cls_)
    {
        if (c->opt.timing) {
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            cudaEventRecord(a, c->stream);
        }
    }
    void done(int nlaunch)
    {
        c->launches += nlaunch;
        if (c->opt.timing) {
            cudaEventRecord(b, c->stream);
            c->pending.push_back({cls, a, b});
            c->nl[cls] += nlaunch;
            a = b = nullptr;
        }
    }
    ~Timed()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

dg_status check_latched(dg_ctx *c)
{
    // err_h mirrors err_d after the last enqueued copy; caller has synchronised.
    const unsigned e = *c->err_h;
    if (e) {
        *c->err_h = 0;
        cudaMemsetAsync(c->err_d, 0, sizeof(unsigned), c->stream);
        if (e & ERR_TIMEOUT)
            return fail(c, DG_ETIMEOUT, "a tensor-core pipeline wait ran out of its time budget; the "
                        "affected surface values are not valid");
        if (e & ERR_NU_RANGE)
            return fail(c, DG_EUNSUPPORTED,
                        "a candidate's FDOA exceeds 0.2 fs (|dfreq/fs| > 0.2); the correlation "
                        "kernels do not handle it");
        if (e & ERR_BIN_SPACING)
            return fail(c, DG_EUNSUPPORTED,
                        "CDFT: a snapshot's FDOA span is too wide for its chunk (chunk x bin spacing > 4e-2 "
                        "cycles); use a shorter chunk or DIRECT");
        return fail(c, DG_EUNSUPPORTED, "a candidate's lag |D| exceeds 1e9 samples");
    }
    return DG_OK;
}

dg_status ensure(dg_ctx *c, void **p, size_t *cap, size_t bytes)
{
    if (*cap >= bytes && *p) return DG_OK;
    if (*p) CK(c, cudaFreeAsync(*p, c->stream));
    *p = nullptr;
    *cap = 0;
    CK(c, cudaMallocAsync(p, bytes, c->stream));
    *cap = bytes;
    return DG_OK;
}

dg_status push_steps(dg_ctx *c)
{
    if (!c->steps_dirty) return DG_OK;
    for (int k = 0; k < c->K; ++k) {
        c->steps_h[k].y1 = c->steps[k].y1;
        c->steps_h[k].y2 = c->steps[k].y2;
        c->steps_h[k].n = (int)c->steps[k].n;
        c->steps_h[k].fmt = c->steps[k].fmt;
    }
    CK(c, cudaMemcpyAsync(c->steps_d, c->steps_h.data(), sizeof(StepDesc) * c->K,
                          cudaMemcpyHostToDevice, c->stream));
    // steps_h must stay unchanged until that copy has run: it is only
    // rewritten by a later push, which first synchronises.
    CK(c, cudaStreamSynchronize(c->stream));
    c->steps_dirty = false;
    return DG_OK;
}

// Correlation for all snapshots over grid gd (ECEF xyz) into surf [K][G],
// then the ordered sum into out.
// Poll limit of the tensor-core pipeline's waits in every CDFT surface
// launched from now on (0 = the kernels' default); set by
// dg_debug_tc_wait_limit, for tests of the timeout path.
static std::atomic<unsigned> g_tc_wait_polls{0};

dg_status run_surface_cdft(dg_ctx *c, const GridDev &gd, const double *xyz, int64_t G, void *surf, void *out,
                           bool refine);

dg_status run_surface(dg_ctx *c, const GridDev &gd, const double *xyz, int64_t G, void *surf, void *out,
                      bool refine)
{
    if (c->opt.algo == DG_ALGO_CDFT) return run_surface_cdft(c, gd, xyz, G, surf, out, refine);
    dg_status st = push_steps(c);
    if (st != DG_OK) return st;
    bool same_fmt = true;
    for (int k = 1; k < c->K; ++k) same_fmt &= c->steps[k].fmt == c->steps[0].fmt;
    CorrArgs a{};
    a.xyz = xyz;
    a.eph = c->eph;
    a.steps = c->steps_d;
    a.surf = surf;
    a.err = c->err_d;
    a.nrows = gd.nrows;
    a.nlon = gd.nlon;
    a.G = G;
    a.fs = c->fs;
    a.lambda = c->lambda;
    a.delay = c->opt.delay;
    a.acc = c->opt.acc;
    a.prec = c->opt.prec;
    a.rows = c->opt.rows;
    const size_t esz = c->opt.prec == DG_PREC_FP64 ? 8 : 4;
    {
        Timed t(c, refine ? DG_K_REFINE : DG_K_CORR);
        if (same_fmt) {
            a.K = c->K;
            a.fmt = c->steps[0].fmt;
            CK(c, launch_corr_direct(a, c->stream));
            t.done(1);
        } else {
            for (int k = 0; k < c->K; ++k) {
                CorrArgs b = a;
                b.K = 1;
                b.fmt = c->steps[k].fmt;
                b.eph = c->eph + 12 * (size_t)k;
                b.steps = c->steps_d + k;
                b.surf = (char *)surf + esz * (size_t)G * k;
                CK(c, launch_corr_direct(b, c->stream));
            }
            t.done(c->K);
        }
    }
    {
        Timed t(c, refine ? DG_K_REFINE : DG_K_ACCUM);
        CK(c, launch_accumulate(surf, c->K, G, c->opt.prec, out, c->stream));
        t.done(1);
    }
    CK(c, cudaMemcpyAsync(c->err_h, c->err_d, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    return DG_OK;
}


template <typename P>
dg_status grow(dg_ctx *c, P **p, size_t n)
{
    if (*p) CK(c, cudaFreeAsync(*p, c->stream));
    *p = nullptr;
    CK(c, cudaMallocAsync((void **)p, sizeof(P) * (n ? n : 1), c->stream));
    return DG_OK;
}


// ---------------------------------------------------------------------------
// Host-side planning for the chunked-DFT surface. Nothing here reads device
// results: every size is an upper bound known from the grid and the
// ephemerides, so the device work of a surface is one stream of launches with
// no host synchronisation (and can be captured in a CUDA graph).
// ---------------------------------------------------------------------------

// Lag slots of snapshot k over a grid of diameter diam (metres). By the
// triangle inequality |rho2 - rho1| <= |p2 - p1|, so |D| <= |p2 - p1| fs / c;
// and each range moves by at most the displacement of the candidate, so D
// varies by at most 2 diam fs / c over the grid. Eq. 9 then gives at most
// 2 ceil(bound) + 1 lags; 2 more absorb rounding, and 3 more the stencil of
// the Lagrange4 delay (lags L - 1 .. L + 2 around floor(D)).
static int lag_slots(const dg_ephem &e, double fs, double diam)
{
    const double dx = e.p2[0] - e.p1[0], dy = e.p2[1] - e.p1[1], dz = e.p2[2] - e.p1[2];
    const double span = std::min(2.0 * std::sqrt(dx * dx + dy * dy + dz * dz), 2.0 * diam) * fs / kC;
    return (int)std::ceil(span) + 6;
}

// FP64 WGS-84 node position and Eq. 3-10 FDOA on the host (planning only).
static void host_node_ecef(const GridDev &g, double i, double j, double p[3])
{
    const double e2 = kF * (2.0 - kF);
    const double s0 = std::sin(g.lat0_rad), w = std::sqrt(1.0 - e2 * s0 * s0);
    const double mr = kA * (1.0 - e2) / (w * w * w), nr = kA / w;
    const double lat = g.lat0_rad + (i - 0.5 * (g.nlat - 1)) * (g.dlat_m / mr);
    const double lon = g.lon0_rad + (j - 0.5 * (g.nlon - 1)) * (g.dlon_m / (nr * std::cos(g.lat0_rad)));
    const double sl = std::sin(lat), n = kA / std::sqrt(1.0 - e2 * sl * sl);
    p[0] = n * std::cos(lat) * std::cos(lon);
    p[1] = n * std::cos(lat) * std::sin(lon);
    p[2] = n * (1.0 - e2) * sl;
}

static double host_nu(const double p[3], const dg_ephem &e, double fs, double lambda)
{
    double f[2];
    for (int r = 0; r < 2; ++r) {
        const double *pp = r ? e.p2 : e.p1, *vv = r ? e.v2 : e.v1;
        const double x = pp[0] - p[0], y = pp[1] - p[1], z = pp[2] - p[2];
        f[r] = -(x * vv[0] + y * vv[1] + z * vv[2]) / (std::sqrt(x * x + y * y + z * z) * lambda);
    }
    return (f[1] - f[0]) / fs;
}

// Diameter bound of the shard: the largest distance between its corners and
// edge midpoints (the grid is a lat/lon rectangle), with a 10 % margin.
static double grid_diameter(const GridDev &g)
{
    double p[9][3];
    int n = 0;
    const double r0 = g.row0, r1 = g.row0 + g.nrows - 1, c1 = g.nlon - 1;
    const double is[3] = {r0, std::round(0.5 * (r0 + r1)), r1}, js[3] = {0.0, std::round(0.5 * c1), c1};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) host_node_ecef(g, is[a], js[b], p[n++]);
    double d = 0.0;
    for (int a = 0; a < n; ++a)
        for (int b = a + 1; b < n; ++b)
            d = std::max(d, std::sqrt((p[a][0] - p[b][0]) * (p[a][0] - p[b][0]) + (p[a][1] - p[b][1]) * (p[a][1] - p[b][1]) +
                                      (p[a][2] - p[b][2]) * (p[a][2] - p[b][2])));
    return 1.1 * d + 1.0;
}

// FDOA span of every snapshot over the shard, from a lattice of nodes (its
// corners, edges and interior; the FDOA field is smooth at these scales): up
// to 65 x 65 nodes, fewer on small shards (at least 9 x 9, about one lattice
// node per 8 grid nodes), the node positions computed once for all
// snapshots.
static void fdoa_spans(const dg_ctx *c, const GridDev &g, std::vector<double> &span,
                       std::vector<double> *lags = nullptr)
{
    const int side = std::max(g.nrows, g.nlon);
    const int lattice = std::min(65, std::max(9, side / 8 + 1));
    const int ni = std::min(lattice, g.nrows), nj = std::min(lattice, g.nlon);
    std::vector<double> p(3 * (size_t)ni * nj);
    for (int a = 0; a < ni; ++a)
        for (int b = 0; b < nj; ++b) {
            const double i = g.row0 + (ni > 1 ? (double)a * (g.nrows - 1) / (ni - 1) : 0.0);
            const double j = nj > 1 ? (double)b * (g.nlon - 1) / (nj - 1) : 0.0;
            host_node_ecef(g, std::round(i), std::round(j), &p[3 * ((size_t)a * nj + b)]);
        }
    span.assign(c->K, 0.0);
    if (lags) lags->assign(c->K, 1.0);
    for (int k = 0; k < c->K; ++k) {
        double lo = 1e300, hi = -1e300, dlo = 1e300, dhi = -1e300;
        const dg_ephem &e = c->eph_host[k];
        for (size_t q = 0; q < (size_t)ni * nj; ++q) {
            const double *x = &p[3 * q];
            const double nu = host_nu(x, e, c->fs, c->lambda);
            lo = std::min(lo, nu);
            hi = std::max(hi, nu);
            if (lags) {  // Eq. 7 and 9: the lattice's lag range
                double r[2];
                for (int t = 0; t < 2; ++t) {
                    const double *pp = t ? e.p2 : e.p1;
                    r[t] = std::sqrt((pp[0] - x[0]) * (pp[0] - x[0]) + (pp[1] - x[1]) * (pp[1] - x[1]) +
                                     (pp[2] - x[2]) * (pp[2] - x[2]));
                }
                const double D = (r[1] - r[0]) * c->fs / kC;
                dlo = std::min(dlo, D);
                dhi = std::max(dhi, D);
            }
        }
        span[k] = hi - lo;
        if (lags) (*lags)[k] = std::floor(dhi + 0.5) - std::floor(dlo + 0.5) + 1.0;
    }
}

// Chunk of a batch with chunk = 0: the longest power of two in
// [64, kCdftAutoMaxChunk] (tensor cores: [64, kCdftAutoMaxChunkTc]) whose
// length times the estimated bin spacing stays within kCdftMDelta / 1.1 (a
// margin for the lattice estimate; the plan kernel checks the bound against
// the exact spacing). On the tensor cores a chunk above kCdftAutoMaxChunk is
// kept only while it fits every capture of the batch and the batch still
// has kCdftMinTilesPerSm lag tiles (128 lags x one chunk, from the lattice's
// lag counts) per SM: longer chunks mean fewer per-lag DFT rows to write and
// to merge into super-chunks, but fewer and longer tiles.
static int auto_chunk(const dg_ctx *c, const std::vector<double> &span, const std::vector<double> &lags, int k0,
                      int S, bool tc)
{
    double dmax = 0.0;
    int64_t nmin = INT64_MAX;
    for (int s = 0; s < S; ++s) {
        dmax = std::max(dmax, span[k0 + s] * (1.0 + 1e-5) / kCdftBinSpan);
        nmin = std::min<int64_t>(nmin, c->steps[k0 + s].n);
    }
    int M = tc ? kCdftAutoMaxChunkTc : kCdftAutoMaxChunk;
    while (M > 64 && 1.1 * M * dmax > kCdftMDelta) M >>= 1;
    auto tiles = [&](int m) {
        double t = 0.0;
        for (int s = 0; s < S; ++s)
            t += std::ceil((double)c->steps[k0 + s].n / m) * std::ceil(lags[k0 + s] / 128.0);
        return t;
    };
    while (M > kCdftAutoMaxChunk && (M > nmin || tiles(M) < (double)kCdftMinTilesPerSm * c->sm_count)) M >>= 1;
    return M;
}

// The batches of a surface and their bucket / combine-group bases: static for
// a grid size G (the main grid and the refinement grid each keep one).
static dg_status cdft_layout(dg_ctx *c, const GridDev &gd, int64_t G, CdftLayout &L)
{
    const double diam = grid_diameter(gd);
    if (L.G == G && L.diam >= diam && !L.batches.empty()) return DG_OK;
    int *old_bb = L.bbase, *old_gb = L.gbase;
    L = CdftLayout{};
    L.G = G;
    L.diam = diam;
    L.bbase = old_bb;
    L.gbase = old_gb;
    // snapshots per batch: per-candidate arrays (16 B per candidate) and the
    // per-lag DFTs (lag slots x chunks x 512 B, chunks at the longest
    // automatic chunk unless one is fixed) within the scratch target
    const double budget = (double)(c->opt.scratch_mib ? c->opt.scratch_mib : 12288) * 1048576.0;
    int64_t nmax = 1;
    int slots_max = 1;
    for (int k = 0; k < c->K; ++k) {
        nmax = std::max<int64_t>(nmax, c->steps[k].n);
        slots_max = std::max(slots_max, lag_slots(c->eph_host[k], c->fs, diam));
    }
    const int m_est = c->opt.chunk ? c->opt.chunk : kCdftAutoMaxChunk;
    const double per_snap = 16.0 * (double)G + (double)slots_max * (double)((nmax + m_est - 1) / m_est) * 512.0;
    int s_max = (int)std::max<int64_t>(1, std::min<int64_t>(c->K, (int64_t)(budget / per_snap)));
    if (c->opt.contract != DG_CONTRACT_FP32) s_max = std::min(s_max, kTcMaxSnapshots);
    std::vector<int> bb, gb;
    for (int k0 = 0; k0 < c->K;) {
        int S = 1;  // same format, at most s_max snapshots
        while (k0 + S < c->K && S < s_max && c->steps[k0 + S].fmt == c->steps[k0].fmt) ++S;
        CdftLayout::Batch t{k0, S, (int)bb.size(), 0, 0};
        int64_t nb = 0, ng = 0;
        for (int s = 0; s <= S; ++s) {
            bb.push_back((int)nb);
            gb.push_back((int)ng);
            if (s == S) break;
            const int slots = lag_slots(c->eph_host[k0 + s], c->fs, diam);
            nb += slots;
            ng += G / kCdftCombineGroup + slots + 1;
        }
        if (nb > INT_MAX / 64 || ng > INT_MAX)
            return fail(c, DG_EUNSUPPORTED, "CDFT: %lld lag slots in one batch; use DIRECT", (long long)nb);
        t.nbt = nb;
        t.groups = ng;
        L.batches.push_back(t);
        L.s_max = std::max(L.s_max, S);
        L.nbt_max = std::max<int64_t>(L.nbt_max, nb);
        L.groups_max = std::max<int64_t>(L.groups_max, ng);
        k0 += S;
    }
    dg_status st;
    if ((st = grow(c, &L.bbase, bb.size())) != DG_OK) return st;
    if ((st = grow(c, &L.gbase, gb.size())) != DG_OK) return st;
    // pageable sources: staged before the calls return
    CK(c, cudaMemcpyAsync(L.bbase, bb.data(), sizeof(int) * bb.size(), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(L.gbase, gb.data(), sizeof(int) * gb.size(), cudaMemcpyHostToDevice, c->stream));
    return DG_OK;
}

// Chunked-DFT surface. Per batch of snapshots (same IQ format, scratch
// within the context's target): geometry, plan (sort by lag
// bucket and bin, bins, tiles), DFT tables, contraction, super-chunks,
// combine. Then the ordered sum. No host synchronisation.
// The ephemerides as double-float (hi, lo) pairs on the device, [K][24].
static dg_status ensure_ephf(dg_ctx *c)
{
    CdftBufs &b = c->cd;
    if (b.ephf_cap >= (size_t)c->K) return DG_OK;
    dg_status st;
    if ((st = grow(c, &b.ephf, 24 * (size_t)c->K)) != DG_OK) return st;
    b.ephf_cap = (size_t)c->K;
    std::vector<float> ef(24 * (size_t)c->K);
    for (int k = 0; k < c->K; ++k) {
        const double *v = &c->eph_host[k].p1[0];
        for (int t = 0; t < 12; ++t) {
            ef[24 * k + 2 * t] = (float)v[t];
            ef[24 * k + 2 * t + 1] = (float)(v[t] - (double)ef[24 * k + 2 * t]);
        }
    }
    // pageable source: staged before the call returns
    CK(c, cudaMemcpyAsync(b.ephf, ef.data(), sizeof(float) * ef.size(), cudaMemcpyHostToDevice, c->stream));
    return DG_OK;
}

// The phases of one chunked-DFT surface: setup (layout, chunks, buffers,
// the candidates' double-float split), then per batch of snapshots its
// arguments, plan, contraction and combine, then the ordered accumulation.
// run_surface_cdft runs them in order; a batch of contexts captured as one
// graph (dg_batch_capture) runs the contraction of the r-th batch of every
// context as one persistent launch between the plans and the combines.
static dg_status cdft_setup(dg_ctx *c, CdftRun &r)
{
    const GridDev &gd = r.gd;
    const double *xyz = r.xyz;
    const int64_t G = r.G;
    const bool refine = r.refine;
    dg_status st = push_steps(c);
    if (st != DG_OK) return st;
    for (int k = 0; k < c->K; ++k)
        if (c->steps[k].n > (1 << 24))
            return fail(c, DG_EUNSUPPORTED, "CDFT: snapshots longer than 2^24 samples are not supported; use DIRECT");
    CdftBufs &b = c->cd;
    CdftLayout &L = refine ? b.loc_layout : b.main_layout;
    r.L = &L;
    // a refinement grid is planned from its shape only (as if centred on the
    // main grid's centre), so that a step captured in a CUDA graph, whose
    // refinement centre is known on the device only, plans it alike
    GridDev shape = gd;
    if (refine) {
        shape.lat0_rad = c->gd.lat0_rad;
        shape.lon0_rad = c->gd.lon0_rad;
    }
    if ((st = cdft_layout(c, shape, G, L)) != DG_OK) return st;
    const int s_max = L.s_max;
    // FDOA spans for the automatic chunk, from the main grid (a refinement
    // grid lies around one of its nodes and spans far less)
    std::vector<double> &span = b.main_span;
    const bool mma = c->opt.contract != DG_CONTRACT_FP32;
    r.mma = mma;
    if (c->opt.chunk == 0 && (span.size() != (size_t)c->K || b.main_lags.size() != (size_t)c->K))
        fdoa_spans(c, c->gd, span, &b.main_lags);
    std::vector<int> &Ms = r.Ms;
    Ms.assign(L.batches.size(), 0);
    int M_max = 64, B_max = 1;
    for (size_t i = 0; i < L.batches.size(); ++i) {
        const auto &t = L.batches[i];
        // Hankel tiles take chunks of at most kLagTileMaxChunk
        const bool tc = mma && c->opt.tiles != DG_TILES_HANKEL;
        Ms[i] = c->opt.chunk ? c->opt.chunk : auto_chunk(c, span, b.main_lags, t.k0, t.S, tc);
        if (refine && !c->opt.chunk) Ms[i] = std::min(Ms[i], kCdftRefineMaxChunk);
        M_max = std::max(M_max, Ms[i]);
        for (int s = 0; s < t.S; ++s) B_max = std::max<int>(B_max, (int)((c->steps[t.k0 + s].n + Ms[i] - 1) / Ms[i]));
    }
    // scratch, grown on demand (never inside a captured graph: a graph is
    // captured after one uncaptured call of the same shape)
    if (b.s_cap < (size_t)s_max) {
        if ((st = grow(c, &b.lr, 2 * (size_t)s_max)) != DG_OK) return st;
        if ((st = grow(c, &b.delta, (size_t)s_max)) != DG_OK) return st;
        if ((st = grow(c, &b.nubase, (size_t)s_max)) != DG_OK) return st;
        if ((st = grow(c, &b.nur, 2 * (size_t)s_max)) != DG_OK) return st;
        if ((st = grow(c, &b.tbase, (size_t)s_max + 1)) != DG_OK) return st;
        if ((st = grow(c, &b.hbase, (size_t)s_max + 1)) != DG_OK) return st;
        if ((st = grow(c, &b.layout, (size_t)s_max)) != DG_OK) return st;
        if ((st = grow(c, &b.Mcs, (size_t)s_max)) != DG_OK) return st;
        b.s_cap = (size_t)s_max;
    }
    if (!b.work) {
        if ((st = grow(c, &b.work, 2)) != DG_OK) return st;
    }
    if (b.sg_cap < (size_t)s_max * G) {
        if ((st = grow(c, &b.candL, (size_t)s_max * G)) != DG_OK) return st;
        if ((st = grow(c, &b.candNu, (size_t)s_max * G)) != DG_OK) return st;
        if ((st = grow(c, &b.order, (size_t)s_max * G)) != DG_OK) return st;
        if ((st = grow(c, &b.nuS, (size_t)s_max * G)) != DG_OK) return st;
        b.sg_cap = (size_t)s_max * G;
    }
    if (c->opt.delay != DG_DELAY_INTEGER && b.mu_cap < (size_t)s_max * G) {
        if ((st = grow(c, &b.candMu, (size_t)s_max * G)) != DG_OK) return st;
        if ((st = grow(c, &b.muS, (size_t)s_max * G)) != DG_OK) return st;
        b.mu_cap = (size_t)s_max * G;
    }
    if (!mma && b.v_cap < (size_t)s_max * M_max * 64) {  // the FP32 contraction's DFT table
        if ((st = grow(c, &b.V, (size_t)s_max * M_max * 64)) != DG_OK) return st;
        b.v_cap = (size_t)s_max * M_max * 64;
    }
    if (b.nb_cap < (size_t)L.nbt_max) {
        const size_t n = (size_t)L.nbt_max;
        if ((st = grow(c, &b.count, n)) != DG_OK) return st;
        if ((st = grow(c, &b.need, n)) != DG_OK) return st;
        if ((st = grow(c, &b.offs, n)) != DG_OK) return st;
        if ((st = grow(c, &b.subcnt, n)) != DG_OK) return st;
        b.nb_cap = n;
    }
    const size_t w_elems = (size_t)L.nbt_max * (size_t)B_max * 128;
    if (w_elems * sizeof(float) > ((size_t)64 << 30))
        return fail(c, DG_EUNSUPPORTED, "CDFT: the per-lag DFT buffer would exceed 64 GiB (%lld lag slots x %d chunks); "
                    "use a longer chunk or DIRECT", (long long)L.nbt_max, B_max);
    if (b.w_cap < w_elems) {
        if ((st = grow(c, &b.W, w_elems)) != DG_OK) return st;
        b.w_cap = w_elems;
    }
    if (b.g2b_cap < (size_t)L.groups_max) {
        if ((st = grow(c, &b.g2b, (size_t)L.groups_max)) != DG_OK) return st;
        b.g2b_cap = (size_t)L.groups_max;
    }
    if (mma) {
        const size_t bt = (size_t)s_max * cdft_btab_bytes(c->opt.contract, M_max);
        if (b.btab_cap < bt) {
            unsigned char *p = reinterpret_cast<unsigned char *>(b.btab);
            if ((st = grow(c, &p, bt)) != DG_OK) return st;
            b.btab = p;
            b.btab_cap = bt;
        }
    }
    const int kplan = refine ? DG_K_REFINE : DG_K_CDFT_PLAN;
    if (!refine) {
        CK(c, cudaMemsetAsync(b.work, 0, 2 * sizeof(unsigned long long), c->stream));
        c->cd_chunk_min = INT_MAX;
        c->cd_chunk_max = 0;
    }
    if ((st = ensure_ephf(c)) != DG_OK) return st;
    if (b.xyzf_cap < (size_t)G) {
        if ((st = grow(c, &b.xyzf, 6 * (size_t)G)) != DG_OK) return st;
        b.xyzf_cap = (size_t)G;
    }
    {
        Timed t(c, kplan);
        CK(c, launch_ecef_split(xyz, G, b.xyzf, c->stream));
        t.done(1);
    }
    if (!refine) c->cd.main_run = r;
    return DG_OK;
}

static void cdft_args(dg_ctx *c, const CdftRun &r, size_t bi, CdftBatch &a)
{
    CdftBufs &b = c->cd;
    const CdftLayout &L = *r.L;
    const std::vector<int> &Ms = r.Ms;
    const bool mma = r.mma, refine = r.refine;
    const double *xyz = r.xyz;
    const GridDev &gd = r.gd;
    const int64_t G = r.G;
    // constants of the geometry as double-float (hi, lo) pairs
    auto split = [](double d, float &h, float &l) {
        h = (float)d;
        l = (float)(d - (double)h);
    };
    const auto &bt = L.batches[bi];
    const int k0 = bt.k0, S = bt.S, M = Ms[bi];
    int Bmax = 1;
    for (int s = 0; s < S; ++s) Bmax = std::max<int>(Bmax, (int)((c->steps[k0 + s].n + M - 1) / M));
    if (!refine) {
        c->cd_chunk_min = std::min(c->cd_chunk_min, M);
        c->cd_chunk_max = std::max(c->cd_chunk_max, M);
    }
    a.xyz = xyz;
    a.xyzf = b.xyzf;
    a.ephf = b.ephf + 24 * (size_t)k0;
    split(c->fs / kC, a.fsc_hi, a.fsc_lo);
    split(1.0 / (c->lambda * c->fs), a.ilf_hi, a.ilf_lo);
    a.eph = c->eph + 12 * (size_t)k0;
    a.sd = c->steps_d + k0;
    a.S = S;
    a.k0 = k0;
    a.G = G;
    a.nrows = gd.nrows;
    a.nlon = gd.nlon;
    a.fs = c->fs;
    a.lambda = c->lambda;
    a.M = M;
    a.Bmax = Bmax;
    a.acc = c->opt.acc;
    a.err = c->err_d;
    a.lr = b.lr;
    a.nur = b.nur;
    a.nubase = b.nubase;
    a.bbase = L.bbase + bt.base;
    a.gbase = L.gbase + bt.base;
    a.candL = b.candL;
    a.candNu = b.candNu;
    a.order = b.order;
    a.nuS = b.nuS;
    a.g2b = b.g2b;
    a.delta = b.delta;
    a.V = b.V;
    a.count = b.count;
    a.need = b.need;
    a.delay = c->opt.delay;
    a.candMu = b.candMu;
    a.muS = b.muS;
    a.offs = b.offs;
    a.subcnt = b.subcnt;
    a.W = b.W;
    a.tbase = b.tbase;
    a.hbase = b.hbase;
    a.layout = b.layout;
    a.Mcs = b.Mcs;
    a.work = refine ? nullptr : b.work;
    a.tiles_mode = c->opt.tiles;
    a.mma = mma ? 1 : 0;
    a.ngroups = (int)bt.groups;
    a.btab = b.btab;
    // FP16 needs the lag products inside its range: int16 products reach 2^31
    const int f = c->steps[k0].fmt;
    const bool fp16 = c->opt.contract == DG_CONTRACT_FP16 || c->opt.contract == DG_CONTRACT_FP16X3;
    a.zscale = (mma && fp16 && f == DG_IQ_CI16) ? 1.0f / 65536.0f : 1.0f;
    a.wait_polls = g_tc_wait_polls.load(std::memory_order_relaxed);
}

static dg_status cdft_plan(dg_ctx *c, const CdftRun &r, const CdftBatch &a, size_t bi)
{
    CdftBufs &b = c->cd;
    const auto &bt = r.L->batches[bi];
    const bool mma = r.mma;
    const int kplan = r.refine ? DG_K_REFINE : DG_K_CDFT_PLAN;
    {
        Timed t(c, kplan);
        CK(c, launch_cdft_geo(a, c->stream));
        CK(c, cudaMemsetAsync(b.g2b, 0xff, sizeof(int4) * (size_t)bt.groups, c->stream));
        CK(c, launch_cdft_plan(a, (int)bt.nbt, c->stream));
        CK(c, launch_cdft_tiles(a, c->stream));
        t.done(mma ? 6 : 7);
    }
    return DG_OK;
}

// The batch's contraction; btab_only: only the tensor cores' DFT operand
// tables (the contraction itself then runs in a launch shared by several
// contexts).
static dg_status cdft_contract(dg_ctx *c, const CdftRun &r, const CdftBatch &a, size_t bi, bool btab_only)
{
    CdftBufs &b = c->cd;
    const auto &bt = r.L->batches[bi];
    const int k0 = bt.k0, S = bt.S, M = r.Ms[bi];
    const bool mma = r.mma, refine = r.refine;
    const CdftLayout &L = *r.L;
    const int f = c->steps[k0].fmt;
    if (btab_only) {
        Timed t(c, refine ? DG_K_REFINE : DG_K_CDFT_CONTRACT);
        CK(c, launch_cdft_btab(a, c->opt.contract, b.btab, c->stream));
        t.done(1);
        return DG_OK;
    }
    {
        Timed t(c, refine ? DG_K_REFINE : DG_K_CDFT_CONTRACT);
        if (mma) {
            // persistent: one CTA per SM, or fewer when the batch can
            // have fewer tiles (the bound: lag tiles of every lag slot)
            int64_t tiles_cap = 0;
            for (int s = 0; s < S; ++s) {
                const int slots = lag_slots(c->eph_host[k0 + s], c->fs, L.diam);
                const int64_t B = (c->steps[k0 + s].n + M - 1) / M;
                tiles_cap += B * ((slots + 127) / 128);
            }
            const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles_cap, c->sm_count));
            // Hankel tiles (chunk <= 1024, on request) run in their own
            // persistent kernel
            const bool hk = M <= kLagTileMaxChunk && c->opt.tiles == DG_TILES_HANKEL;
            int n = 0;
            if (c->opt.tiles != DG_TILES_HANKEL || M > kLagTileMaxChunk) {
                CK(c, launch_cdft_btab(a, c->opt.contract, b.btab, c->stream));
                CK(c, launch_cdft_contract_mma(a, grid, f, c->opt.contract, c->stream));
                n += 2;
            }
            if (hk) {
                int64_t hk_cap = 0;
                for (int s = 0; s < S; ++s) {
                    const int slots = lag_slots(c->eph_host[k0 + s], c->fs, L.diam);
                    const int64_t B = (c->steps[k0 + s].n + M - 1) / M;
                    hk_cap += B * ((slots + kHkLags - 1) / kHkLags);
                }
                const int hgrid = (int)std::max<int64_t>(1, std::min<int64_t>(hk_cap, c->sm_count));
                CK(c, launch_cdft_contract_hankel(a, hgrid, f, c->opt.contract, c->stream));
                ++n;
            }
            t.done(n);
        } else {
            CK(c, launch_cdft_contract_fp32(a, (int)bt.nbt, f, c->stream));
            t.done(1);
        }
    }
    return DG_OK;
}

static dg_status cdft_combine(dg_ctx *c, const CdftRun &r, const CdftBatch &a, size_t bi)
{
    const auto &bt = r.L->batches[bi];
    const bool refine = r.refine;
    float *surf_f = reinterpret_cast<float *>(r.surf);
    {
        Timed t(c, refine ? DG_K_REFINE : DG_K_CDFT_COMBINE);
        CK(c, launch_cdft_superchunk(a, (int)bt.nbt, c->stream));
        CK(c, launch_cdft_combine(a, surf_f, c->stream));
        t.done(2);
    }
    return DG_OK;
}

static dg_status cdft_finish(dg_ctx *c, const CdftRun &r)
{
    const bool refine = r.refine;
    {
        Timed t(c, refine ? DG_K_REFINE : DG_K_ACCUM);
        CK(c, launch_accumulate(r.surf, c->K, r.G, DG_PREC_FP32, r.out, c->stream));
        t.done(1);
    }
    CK(c, cudaMemcpyAsync(c->err_h, c->err_d, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    return DG_OK;
}


dg_status run_surface_cdft(dg_ctx *c, const GridDev &gd, const double *xyz, int64_t G, void *surf, void *out,
                           bool refine)
{
    CdftRun r;
    r.gd = gd;
    r.xyz = xyz;
    r.G = G;
    r.surf = surf;
    r.out = out;
    r.refine = refine;
    dg_status st = cdft_setup(c, r);
    if (st != DG_OK) return st;
    for (size_t bi = 0; bi < r.L->batches.size(); ++bi) {
        CdftBatch a{};
        cdft_args(c, r, bi, a);
        if ((st = cdft_plan(c, r, a, bi)) != DG_OK) return st;
        if ((st = cdft_contract(c, r, a, bi, false)) != DG_OK) return st;
        if ((st = cdft_combine(c, r, a, bi)) != DG_OK) return st;
    }
    return cdft_finish(c, r);
}

dg_status run_argmax(dg_ctx *c, const void *v, int64_t n, const GridDev &gd, ArgmaxResult *host)
{
    size_t need = argmax_tmp_bytes(n);
    dg_status st = ensure(c, &c->amax_tmp, &c->amax_tmp_bytes, need);
    if (st != DG_OK) return st;
    int nlaunch = 0;
    {
        Timed t(c, DG_K_ARGMAX);
        CK(c, launch_argmax(v, n, c->opt.prec, gd, c->amax_tmp, c->amax_res, &nlaunch, c->stream));
        t.done(nlaunch);
    }
    CK(c, cudaMemcpyAsync(c->amax_host, c->amax_res, sizeof(ArgmaxResult), cudaMemcpyDeviceToHost,
                          c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    *host = *c->amax_host;
    return DG_OK;
}

GridDev make_griddev(const dg_grid &g, int row0, int nrows)
{
    GridDev d;
    d.lat0_rad = g.lat0_deg * (kPi / 180.0);
    d.lon0_rad = g.lon0_deg * (kPi / 180.0);
    d.dlat_m = g.dlat_m;
    d.dlon_m = g.dlon_m;
    d.nlat = g.nlat;
    d.nlon = g.nlon;
    d.row0 = row0;
    d.nrows = nrows;
    return d;
}

dg_status validate_grid(dg_ctx *c, const dg_grid *g)
{
    if (!g) return fail(c, DG_EINVAL, "grid is NULL");
    if (!(std::isfinite(g->lat0_deg) && std::fabs(g->lat0_deg) < 89.0))
        return fail(c, DG_EINVAL, "lat0_deg must be finite and within +-89 deg");
    if (!std::isfinite(g->lon0_deg)) return fail(c, DG_EINVAL, "lon0_deg must be finite");
    if (!(g->dlat_m > 0 && g->dlon_m > 0 && std::isfinite(g->dlat_m) && std::isfinite(g->dlon_m)))
        return fail(c, DG_EINVAL, "grid spacing must be positive and finite");
    if (g->nlat < 1 || g->nlon < 1) return fail(c, DG_EINVAL, "nlat and nlon must be >= 1");
    if ((int64_t)g->nlat * g->nlon > (int64_t)1 << 31)
        return fail(c, DG_EUNSUPPORTED, "grid larger than 2^31 nodes");
    return DG_OK;
}

}  // namespace

extern "C" {

int32_t dg_abi_version(void) { return DG_ABI_VERSION; }

void dg_options_default(dg_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->delay = DG_DELAY_INTEGER;
    o->acc = DG_ACC_POWER;
    o->prec = DG_PREC_FP32;
    o->algo = DG_ALGO_DIRECT;
}

const char *dg_last_error(const dg_ctx *ctx) { return ctx ? ctx->err.c_str() : g_thread_error.c_str(); }

dg_status dg_create(const dg_grid *grid, const dg_ephem *eph, int32_t K, double fs_hz, double fc_hz,
                    const dg_options *opt, void *cuda_stream, dg_ctx **out)
{
    g_thread_error.clear();
    if (!out) return fail(nullptr, DG_EINVAL, "out is NULL");
    dg_status st = validate_grid(nullptr, grid);
    if (st != DG_OK) return st;
    if (!eph) return fail(nullptr, DG_EINVAL, "eph is NULL");
    if (K < 1 || K > 65535) return fail(nullptr, DG_EINVAL, "K must be in [1, 65535]");
    if (!(fs_hz > 0 && std::isfinite(fs_hz))) return fail(nullptr, DG_EINVAL, "fs_hz must be > 0");
    if (!(fc_hz > 0 && std::isfinite(fc_hz))) return fail(nullptr, DG_EINVAL, "fc_hz must be > 0");
    dg_options o;
    dg_options_default(&o);
    if (opt) o = *opt;
    if (o.delay != DG_DELAY_INTEGER && o.delay != DG_DELAY_LAGRANGE4)
        return fail(nullptr, DG_EINVAL, "unknown delay mode %d", o.delay);
    if (o.acc != DG_ACC_POWER && o.acc != DG_ACC_MAG) return fail(nullptr, DG_EINVAL, "unknown acc mode %d", o.acc);
    if (o.prec != DG_PREC_FP32 && o.prec != DG_PREC_FP64)
        return fail(nullptr, DG_EINVAL, "unknown precision %d", o.prec);
    if (o.algo != DG_ALGO_DIRECT && o.algo != DG_ALGO_CDFT) return fail(nullptr, DG_EINVAL, "unknown algorithm %d", o.algo);
    if (o.algo == DG_ALGO_CDFT) {
        if (o.prec != DG_PREC_FP32) return fail(nullptr, DG_EUNSUPPORTED, "CDFT writes FP32 surfaces only");
        if (o.chunk != 0 && (o.chunk < 64 || o.chunk > kCdftMaxChunk || o.chunk % 64 != 0))
            return fail(nullptr, DG_EINVAL, "chunk must be 0 or a multiple of 64 in [64, %d]", kCdftMaxChunk);
        if (o.bins != 0 && o.bins != 64) return fail(nullptr, DG_EUNSUPPORTED, "bins must be 0 or 64");
        if (o.contract < DG_CONTRACT_FP32 || o.contract > DG_CONTRACT_FP16X3)
            return fail(nullptr, DG_EINVAL, "unknown contraction arithmetic %d", o.contract);
        if (o.tiles < DG_TILES_AUTO || o.tiles > DG_TILES_HANKEL)
            return fail(nullptr, DG_EINVAL, "unknown tile shape %d", o.tiles);
        if (o.tiles == DG_TILES_HANKEL && o.chunk > kLagTileMaxChunk)
            return fail(nullptr, DG_EINVAL, "Hankel tiles need chunk <= %d", kLagTileMaxChunk);
        if (o.tiles == DG_TILES_LAGS && o.chunk > kLagTileMaxChunk && o.chunk % kLagTileMaxChunk != 0)
            return fail(nullptr, DG_EINVAL, "lag tiles need chunk <= %d or a multiple of it", kLagTileMaxChunk);
        if (o.scratch_mib < 0) return fail(nullptr, DG_EINVAL, "scratch_mib must be >= 0");
    }
    if (!direct_rows_ok(o.prec, o.rows))
        return fail(nullptr, DG_EINVAL, "rows must be 0, 4, 8 or 16 (FP32) or 0, 2 or 4 (FP64)");
    if (o.row0 < 0 || o.row0 >= grid->nlat) return fail(nullptr, DG_EINVAL, "row0 outside the grid");
    if (o.nrows < 0 || o.row0 + o.nrows > grid->nlat) return fail(nullptr, DG_EINVAL, "row shard outside the grid");
    for (int k = 0; k < K; ++k)
        if (!finite3(eph[k].p1) || !finite3(eph[k].v1) || !finite3(eph[k].p2) || !finite3(eph[k].v2))
            return fail(nullptr, DG_EINVAL, "ephemeris %d is not finite", k);

    dg_ctx *c = new (std::nothrow) dg_ctx();
    if (!c) return fail(nullptr, DG_ENOMEM, "host allocation failed");
    c->grid = *grid;
    c->opt = o;
    c->K = K;
    c->fs = fs_hz;
    c->fc = fc_hz;
    c->lambda = kC / fc_hz;
    c->stream = (cudaStream_t)cuda_stream;
    const int nrows = o.nrows ? o.nrows : grid->nlat - o.row0;
    c->gd = make_griddev(*grid, o.row0, nrows);
    c->G = (int64_t)nrows * grid->nlon;
    c->eph_host.assign(eph, eph + K);
    c->steps.resize(K);
    c->steps_h.resize(K);

    auto bail = [&](dg_status s) {
        g_thread_error = c->err;
        dg_destroy(c);
        return s;
    };
#define CKC(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return bail(fail(c, e_ == cudaErrorMemoryAllocation ? DG_ENOMEM : DG_ECUDA, "%s: %s", \
                             #call, cudaGetErrorString(e_)));                                  \
    } while (0)
    CKC(cudaGetDevice(&c->device));
    CKC(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device));
    CKC(cudaMallocAsync((void **)&c->xyz, sizeof(double) * 3 * (size_t)c->G, c->stream));
    c->xyz_cap = c->G;
    CKC(cudaMallocAsync((void **)&c->eph, sizeof(double) * 12 * (size_t)K, c->stream));
    CKC(cudaMallocAsync((void **)&c->steps_d, sizeof(StepDesc) * (size_t)K, c->stream));
    CKC(cudaMallocAsync((void **)&c->amax_res, sizeof(ArgmaxResult), c->stream));
    CKC(cudaMallocAsync((void **)&c->err_d, sizeof(unsigned), c->stream));
    CKC(cudaMallocHost((void **)&c->amax_host, sizeof(ArgmaxResult)));
    CKC(cudaMallocHost((void **)&c->err_h, sizeof(unsigned)));
    *c->err_h = 0;
    CKC(cudaMemsetAsync(c->err_d, 0, sizeof(unsigned), c->stream));
    CKC(cudaMemcpyAsync(c->eph, c->eph_host.data(), sizeof(dg_ephem) * (size_t)K, cudaMemcpyHostToDevice,
                        c->stream));
    {
        Timed t(c, DG_K_GRID);
        CKC(launch_grid_ecef(c->gd, c->xyz, c->stream));
        t.done(1);
    }
    CKC(cudaStreamSynchronize(c->stream));  // eph_host may not move before the copy ran
#undef CKC
    *out = c;
    return DG_OK;
}

dg_status dg_set_grid(dg_ctx *c, const dg_grid *grid)
{
    if (!c) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    c->err.clear();
    dg_status st = validate_grid(c, grid);
    if (st != DG_OK) return st;
    if (c->gd.row0 != 0 || c->gd.nrows != c->grid.nlat)
        return fail(c, DG_EUNSUPPORTED, "dg_set_grid needs a context over the whole grid (no row shard)");
    const int64_t G = (int64_t)grid->nlat * grid->nlon;
    if (G > c->xyz_cap) {
        CK(c, cudaFreeAsync(c->xyz, c->stream));
        c->xyz = nullptr;
        c->xyz_cap = 0;
        CK(c, cudaMallocAsync((void **)&c->xyz, sizeof(double) * 3 * (size_t)G, c->stream));
        c->xyz_cap = G;
    }
    c->grid = *grid;
    c->opt.row0 = 0;
    c->opt.nrows = 0;
    c->gd = make_griddev(*grid, 0, grid->nlat);
    c->G = G;
    c->cd.main_span.clear();  // FDOA spans and lag counts of the old grid
    c->cd.main_lags.clear();
    ++c->steps_gen;           // graphs and batches recorded on the old grid are stale
    {
        Timed t(c, DG_K_GRID);
        CK(c, launch_grid_ecef(c->gd, c->xyz, c->stream));
        t.done(1);
    }
    return DG_OK;
}

dg_status dg_load_capture(dg_ctx *c, int32_t step, int32_t fmt, const void *y1, const void *y2,
                          int64_t n, int32_t is_device_ptr)
{
    if (!c) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    c->err.clear();
    if (step < 0 || step >= c->K) return fail(c, DG_EINVAL, "step %d outside [0, %d)", step, c->K);
    const size_t bps = iq_bytes(fmt);
    if (!bps) return fail(c, DG_EINVAL, "unknown IQ format %d", fmt);
    if (!y1 || !y2) return fail(c, DG_EINVAL, "y1 and y2 must not be NULL");
    if (n < 1) return fail(c, DG_EINVAL, "n_samples must be >= 1");
    if (n > ((int64_t)1 << 30)) return fail(c, DG_EUNSUPPORTED, "n_samples above 2^30");
    Step &s = c->steps[step];
    const size_t bytes = bps * (size_t)n;
    if (s.cap < bytes) {
        if (s.y1) CK(c, cudaFreeAsync(s.y1, c->stream));
        if (s.y2) CK(c, cudaFreeAsync(s.y2, c->stream));
        s.y1 = s.y2 = nullptr;
        s.cap = 0;
        s.loaded = false;
        CK(c, cudaMallocAsync(&s.y1, bytes, c->stream));
        CK(c, cudaMallocAsync(&s.y2, bytes, c->stream));
        s.cap = bytes;
        ++c->steps_gen;
    }
    const cudaMemcpyKind kind = is_device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(c, cudaMemcpyAsync(s.y1, y1, bytes, kind, c->stream));
    CK(c, cudaMemcpyAsync(s.y2, y2, bytes, kind, c->stream));
    if (s.fmt != fmt || s.n != n || !s.loaded) {
        c->steps_dirty = true;
        ++c->steps_gen;
    }
    s.fmt = fmt;
    s.n = n;
    s.loaded = true;
    return DG_OK;
}

dg_status dg_cost_surface(dg_ctx *c, void *out)
{
    if (!c) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    c->err.clear();
    if (!out) return fail(c, DG_EINVAL, "out is NULL");
    for (int k = 0; k < c->K; ++k)
        if (!c->steps[k].loaded) return fail(c, DG_ESTATE, "snapshot %d has not been loaded", k);
    const size_t esz = c->opt.prec == DG_PREC_FP64 ? 8 : 4;
    dg_status st = ensure(c, &c->surf, &c->surf_bytes, esz * (size_t)c->G * c->K);
    if (st != DG_OK) return st;
    return run_surface(c, c->gd, c->xyz, c->G, c->surf, out, false);
}

dg_status dg_sync(dg_ctx *c)
{
    if (!c) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    c->err.clear();
    CK(c, cudaStreamSynchronize(c->stream));
    return check_latched(c);
}

// Buffers of a refinement grid of G nodes.
static dg_status ensure_local(dg_ctx *c, int64_t G)
{
    const size_t esz = c->opt.prec == DG_PREC_FP64 ? 8 : 4;
    if (c->loc.g_cap < (size_t)G) {
        if (c->loc.xyz) CK(c, cudaFreeAsync(c->loc.xyz, c->stream));
        if (c->loc.surf) CK(c, cudaFreeAsync(c->loc.surf, c->stream));
        if (c->loc.cost) CK(c, cudaFreeAsync(c->loc.cost, c->stream));
        c->loc = LocalGrid{};
        CK(c, cudaMallocAsync((void **)&c->loc.xyz, sizeof(double) * 3 * G, c->stream));
        CK(c, cudaMallocAsync(&c->loc.surf, esz * G * c->K + 8, c->stream));
        CK(c, cudaMallocAsync(&c->loc.cost, esz * G + 8, c->stream));
        c->loc.g_cap = (size_t)G;
    }
    return DG_OK;
}

// Half-width (nodes) of the refinement grid of dg_argmax_refine; 0 = none.
static dg_status refine_half(dg_ctx *c, double spacing_m, double window_m, int *half)
{
    *half = 0;
    if (!(spacing_m > 0 && window_m >= spacing_m)) return DG_OK;
    if (!(std::isfinite(spacing_m) && std::isfinite(window_m)))
        return fail(c, DG_EINVAL, "refinement spacing and window must be finite");
    const double h = std::floor(window_m / spacing_m + 0.5);
    if (h > 2000) return fail(c, DG_EINVAL, "refinement grid wider than 4001 nodes");
    *half = (int)h;
    return DG_OK;
}

dg_status dg_argmax_refine(dg_ctx *c, const void *cost, double spacing_m, double window_m, dg_fix *out)
{
    if (!c) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    c->err.clear();
    if (!cost || !out) return fail(c, DG_EINVAL, "cost and out must not be NULL");
    const bool refine = spacing_m > 0 && window_m >= spacing_m;
    int half = 0;
    if (refine) {
        if (!(std::isfinite(spacing_m) && std::isfinite(window_m)))
            return fail(c, DG_EINVAL, "refinement spacing and window must be finite");
        const double h = std::floor(window_m / spacing_m + 0.5);
        if (h > 2000) return fail(c, DG_EINVAL, "refinement grid wider than 4001 nodes");
        half = (int)h;
    }
    CK(c, cudaStreamSynchronize(c->stream));
    dg_status st = check_latched(c);
    if (st != DG_OK) return st;
    ArgmaxResult r;
    st = run_argmax(c, cost, c->G, c->gd, &r);
    if (st != DG_OK) return st;
    if (r.idx < 0) return fail(c, DG_EINVAL, "the surface holds no finite value");
    dg_fix f;
    std::memset(&f, 0, sizeof f);
    f.index = r.idx;
    f.i = c->gd.row0 + (int)(r.idx / c->gd.nlon);
    f.j = (int)(r.idx % c->gd.nlon);
    f.lat_deg = r.lat_rad * (180.0 / kPi);
    f.lon_deg = r.lon_rad * (180.0 / kPi);
    f.cost = r.val;
    f.sub_lat_deg = r.sub_lat_rad * (180.0 / kPi);
    f.sub_lon_deg = r.sub_lon_rad * (180.0 / kPi);
    if (refine) {
        const int n = 2 * half + 1;
        dg_grid lg;
        lg.lat0_deg = f.lat_deg;
        lg.lon0_deg = f.lon_deg;
        lg.dlat_m = spacing_m;
        lg.dlon_m = spacing_m;
        lg.nlat = n;
        lg.nlon = n;
        const GridDev lgd = make_griddev(lg, 0, n);
        const int64_t G = (int64_t)n * n;
        if ((st = ensure_local(c, G)) != DG_OK) return st;
        {
            Timed t(c, DG_K_REFINE);
            CK(c, launch_grid_ecef(lgd, c->loc.xyz, c->stream));
            t.done(1);
        }
        st = run_surface(c, lgd, c->loc.xyz, G, c->loc.surf, c->loc.cost, true);
        if (st != DG_OK) return st;
        CK(c, cudaStreamSynchronize(c->stream));
        st = check_latched(c);
        if (st != DG_OK) return st;
        ArgmaxResult q;
        st = run_argmax(c, c->loc.cost, G, lgd, &q);
        if (st != DG_OK) return st;
        if (q.idx < 0) return fail(c, DG_EINVAL, "the refinement surface holds no finite value");
        f.refine_n = n;
        f.ri = (int)(q.idx / n);
        f.rj = (int)(q.idx % n);
        f.refined_lat_deg = q.lat_rad * (180.0 / kPi);
        f.refined_lon_deg = q.lon_rad * (180.0 / kPi);
        f.refined_cost = q.val;
        f.sub_lat_deg = q.sub_lat_rad * (180.0 / kPi);
        f.sub_lon_deg = q.sub_lon_rad * (180.0 / kPi);
    }
    *out = f;
    return DG_OK;
}

dg_status dg_detect(dg_ctx *c, const void *cost, double threshold, int32_t relative, int32_t radius,
                    int32_t max_peaks, dg_peak *out, int32_t *n_out)
{
    if (!c) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    c->err.clear();
    if (!cost || !out || !n_out) return fail(c, DG_EINVAL, "cost, out and n_out must not be NULL");
    if (radius < 0 || radius > 64) return fail(c, DG_EINVAL, "radius must be in [0, 64]");
    if (max_peaks < 1 || max_peaks > kDetectCap) return fail(c, DG_EINVAL, "max_peaks must be in [1, %d]", kDetectCap);
    if (!std::isfinite(threshold)) return fail(c, DG_EINVAL, "threshold must be finite");
    constexpr int kCap = kDetectCap;
    CK(c, cudaStreamSynchronize(c->stream));
    dg_status st = check_latched(c);
    if (st != DG_OK) return st;
    double thr = threshold;
    if (relative) {
        ArgmaxResult r;
        if ((st = run_argmax(c, cost, c->G, c->gd, &r)) != DG_OK) return st;
        if (r.idx < 0) return fail(c, DG_EINVAL, "the surface holds no finite value");
        thr = threshold * r.val;
    }
    if (!c->det_count) {
        CK(c, cudaMallocAsync((void **)&c->det_count, sizeof(int), c->stream));
        CK(c, cudaMallocAsync((void **)&c->det_cand, sizeof(int64_t) * kCap, c->stream));
        CK(c, cudaMallocAsync((void **)&c->det_out, sizeof(DetectPeak) * kCap, c->stream));
    }
    int count = 0;
    std::vector<DetectPeak> pk((size_t)max_peaks);
    for (int round = 0;; ++round) {
        {
            Timed t(c, DG_K_ARGMAX);
            CK(c, launch_detect(cost, c->opt.prec, c->gd, thr, radius, kCap, max_peaks, c->det_count, c->det_cand,
                                c->det_out, c->stream));
            t.done(2);
        }
        CK(c, cudaMemcpyAsync(&count, c->det_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaMemcpyAsync(pk.data(), c->det_out, sizeof(DetectPeak) * (size_t)max_peaks, cudaMemcpyDeviceToHost,
                              c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        if (count <= kCap) break;
        // More peaks pass than the sort holds: it ordered kCap of them (an
        // arbitrary subset), so at least max_peaks peaks reach its
        // max_peaks-th value, and so does every one of the max_peaks largest.
        // That value is the next threshold; far fewer peaks pass it.
        const double next = pk[(size_t)max_peaks - 1].value;
        if (!(next > thr) || round >= 8)
            return fail(c, DG_EUNSUPPORTED, "%d peaks of equal value pass the detection test (max %d); raise the "
                        "threshold", count, kCap);
        thr = next;
    }
    const int n = std::min(count, (int)max_peaks);
    for (int k = 0; k < n; ++k) {
        out[k].index = pk[k].index;
        out[k].i = pk[k].i;
        out[k].j = pk[k].j;
        out[k].lat_deg = pk[k].lat_rad * (180.0 / kPi);
        out[k].lon_deg = pk[k].lon_rad * (180.0 / kPi);
        out[k].value = pk[k].value;
    }
    *n_out = n;
    return DG_OK;
}

// ---------------------------------------------------------------------------
// Whole steps as CUDA graphs
// ---------------------------------------------------------------------------

// Buffers a device-only step needs (allocated outside any capture).
static dg_status prepare_step(dg_ctx *c, int half)
{
    for (int k = 0; k < c->K; ++k)
        if (!c->steps[k].loaded) return fail(c, DG_ESTATE, "snapshot %d has not been loaded", k);
    const size_t esz = c->opt.prec == DG_PREC_FP64 ? 8 : 4;
    dg_status st = ensure(c, &c->surf, &c->surf_bytes, esz * (size_t)c->G * c->K);
    if (st != DG_OK) return st;
    const int n = 2 * half + 1;
    const int64_t Gl = half > 0 ? (int64_t)n * n : 0;
    if ((st = ensure(c, &c->amax_tmp, &c->amax_tmp_bytes, argmax_tmp_bytes(std::max<int64_t>(c->G, Gl)))) != DG_OK)
        return st;
    if (half > 0 && (st = ensure_local(c, Gl)) != DG_OK) return st;
    if (!c->amax_fine) CK(c, cudaMallocAsync((void **)&c->amax_fine, sizeof(ArgmaxResult), c->stream));
    if (!c->fix_dev) CK(c, cudaMallocAsync((void **)&c->fix_dev, sizeof(dg_fix), c->stream));
    if (!c->fix_host) CK(c, cudaMallocHost((void **)&c->fix_host, sizeof(dg_fix)));
    return push_steps(c);
}

// One step on the device only: the surface into cost, its argmax, the
// refinement grid centred on it (built on the device), the refinement
// surface and argmax, and the fix record copied to the pinned fix_host. No
// host synchronisation and no allocation (prepare_step ran before).
static dg_status step_device_post(dg_ctx *c, void *cost, double spacing_m, int half);

static dg_status step_device(dg_ctx *c, void *cost, double spacing_m, int half)
{
    dg_status st = run_surface(c, c->gd, c->xyz, c->G, c->surf, cost, false);
    if (st != DG_OK) return st;
    return step_device_post(c, cost, spacing_m, half);
}

// The rest of a step once the surface is enqueued: its argmax, the
// refinement, the fix record.
static dg_status step_device_post(dg_ctx *c, void *cost, double spacing_m, int half)
{
    dg_status st = DG_OK;
    int nl = 0;
    CK(c, launch_argmax(cost, c->G, c->opt.prec, c->gd, c->amax_tmp, c->amax_res, &nl, c->stream));
    const ArgmaxResult *fine = nullptr;
    const int n = 2 * half + 1;
    if (half > 0) {
        dg_grid lg;
        lg.lat0_deg = c->grid.lat0_deg;  // replaced on the device by the argmax node
        lg.lon0_deg = c->grid.lon0_deg;
        lg.dlat_m = lg.dlon_m = spacing_m;
        lg.nlat = lg.nlon = n;
        const GridDev lgd = make_griddev(lg, 0, n);
        const int64_t Gl = (int64_t)n * n;
        CK(c, launch_grid_ecef(lgd, c->loc.xyz, c->stream, c->amax_res));
        ++nl;
        st = run_surface(c, lgd, c->loc.xyz, Gl, c->loc.surf, c->loc.cost, true);
        if (st != DG_OK) return st;
        CK(c, launch_argmax(c->loc.cost, Gl, c->opt.prec, lgd, c->amax_tmp, c->amax_fine, &nl, c->stream,
                            c->amax_res));
        fine = c->amax_fine;
    }
    CK(c, launch_make_fix(c->amax_res, fine, c->gd, half > 0 ? n : 0, c->fix_dev, c->stream));
    ++nl;
    c->launches += nl;
    CK(c, cudaMemcpyAsync(c->fix_host, c->fix_dev, sizeof(dg_fix), cudaMemcpyDeviceToHost, c->stream));
    return DG_OK;
}

static dg_status read_fix(dg_ctx *c, dg_fix *out)
{
    CK(c, cudaStreamSynchronize(c->stream));
    dg_status st = check_latched(c);
    if (st != DG_OK) return st;
    if (c->fix_host->index < 0) return fail(c, DG_EINVAL, "the surface holds no finite value");
    if (c->fix_host->refine_n > 0 && c->fix_host->ri < 0)
        return fail(c, DG_EINVAL, "the refinement surface holds no finite value");
    *out = *c->fix_host;
    return DG_OK;
}

// Capture one step of each context as a branch of one graph: forked from and
// joined to `stream`. Timing is off inside the capture.
// The shared contraction rounds of a batch (dg_batch_capture): round r runs,
// in one persistent launch, the contraction of the r-th snapshot batch of
// every context that has one; each context plans and combines its batch on
// its own stream around it.
struct TcRounds {
    std::vector<std::vector<int>> ctx;  // per round: the contexts taking part
    std::vector<int> job_off;           // per round: its first job in jobs
    std::vector<int> tile_off;          // per round: its prefix sums in job_tiles
    TcJob *jobs = nullptr;              // device, every round's jobs in order
    int *job_tiles = nullptr;           // device, per round n_r + 1 tile prefix sums
    int fmt = 0, contract = 0;
    unsigned wait_polls = 0;
};

// Every context on the tensor-core CDFT path (lag or row tiles), one capture
// format and one contraction arithmetic across all of them: the batch's
// contractions can share launches. The contexts have run one uncaptured
// step, so their layouts and buffers exist. Builds the job tables on the
// device (synchronously, before any capture).
static dg_status tc_rounds(dg_ctx *const *ctxs, int n, TcRounds &R, bool &ok)
{
    ok = false;
    if (n < 2) return DG_OK;
    const int fmt = ctxs[0]->steps[0].fmt, contract = ctxs[0]->opt.contract;
    size_t rounds = 0;
    for (int i = 0; i < n; ++i) {
        dg_ctx *c = ctxs[i];
        if (c->opt.algo != DG_ALGO_CDFT || c->opt.contract == DG_CONTRACT_FP32 || c->opt.tiles == DG_TILES_HANKEL ||
            c->opt.contract != contract || !c->cd.main_run.L)
            return DG_OK;
        for (int k = 0; k < c->K; ++k)
            if (c->steps[k].fmt != fmt) return DG_OK;
        rounds = std::max(rounds, c->cd.main_run.L->batches.size());
    }
    std::vector<TcJob> jobs;
    R.ctx.assign(rounds, {});
    for (size_t r = 0; r < rounds; ++r) {
        R.job_off.push_back((int)jobs.size());
        R.tile_off.push_back((int)(jobs.size() + r));
        for (int i = 0; i < n; ++i) {
            dg_ctx *c = ctxs[i];
            if (r >= c->cd.main_run.L->batches.size()) continue;
            CdftBatch a{};
            cdft_args(c, c->cd.main_run, r, a);
            jobs.push_back(tc_job(a, a.btab));
            R.ctx[r].push_back(i);
        }
    }
    dg_ctx *c0 = ctxs[0];
    CK(c0, cudaMalloc((void **)&R.jobs, sizeof(TcJob) * jobs.size()));
    CK(c0, cudaMalloc((void **)&R.job_tiles, sizeof(int) * (jobs.size() + rounds)));
    CK(c0, cudaMemcpy(R.jobs, jobs.data(), sizeof(TcJob) * jobs.size(), cudaMemcpyHostToDevice));
    R.fmt = fmt;
    R.contract = contract;
    R.wait_polls = g_tc_wait_polls.load(std::memory_order_relaxed);
    ok = true;
    return DG_OK;
}

static void tc_rounds_free(TcRounds &R)
{
    if (R.jobs) cudaFree(R.jobs);
    if (R.job_tiles) cudaFree(R.job_tiles);
    R.jobs = nullptr;
    R.job_tiles = nullptr;
}

// The surfaces of a batch's contexts with shared contraction rounds (inside
// a capture): setup, then per round every context's plan, one launch, every
// context's combine; then each context's accumulation. Returns the shared
// launches in *shared.
static dg_status shared_surfaces(dg_ctx *const *ctxs, int n, void *const *costs, const TcRounds &R,
                                 cudaStream_t stream, int64_t *shared)
{
    dg_ctx *c0 = ctxs[0];
    std::vector<CdftRun> runs((size_t)n);
    for (int i = 0; i < n; ++i) {
        dg_ctx *c = ctxs[i];
        CdftRun &r = runs[(size_t)i];
        r.gd = c->gd;
        r.xyz = c->xyz;
        r.G = c->G;
        r.surf = c->surf;
        r.out = costs[i];
        r.refine = false;
        dg_status st = cdft_setup(c, r);
        if (st != DG_OK) return st;
    }
    std::vector<cudaEvent_t> evs;
    auto event = [&](cudaEvent_t *e) {
        const cudaError_t x = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
        if (x == cudaSuccess) evs.push_back(*e);
        return x;
    };
    dg_status st = DG_OK;
    cudaError_t e = cudaSuccess;
    for (size_t rd = 0; rd < R.ctx.size() && st == DG_OK && e == cudaSuccess; ++rd) {
        const std::vector<int> &part = R.ctx[rd];
        for (int i : part) {
            dg_ctx *c = ctxs[i];
            CdftBatch a{};
            cdft_args(c, runs[(size_t)i], rd, a);
            if ((st = cdft_plan(c, runs[(size_t)i], a, rd)) != DG_OK) break;
            if ((st = cdft_contract(c, runs[(size_t)i], a, rd, true)) != DG_OK) break;
            cudaEvent_t ev;
            if ((e = event(&ev)) != cudaSuccess || (e = cudaEventRecord(ev, c->stream)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(stream, ev, 0)) != cudaSuccess)
                break;
        }
        if (st != DG_OK || e != cudaSuccess) break;
        const int nr = (int)part.size();
        TcJob *jobs = R.jobs + R.job_off[rd];
        int *tiles = R.job_tiles + R.tile_off[rd];
        if ((e = launch_tc_job_tiles(jobs, nr, tiles, stream)) != cudaSuccess) break;
        if ((e = launch_cdft_contract_jobs(jobs, nr, tiles, c0->sm_count, R.fmt, R.contract, R.wait_polls, stream)) !=
            cudaSuccess)
            break;
        *shared += 2;
        cudaEvent_t done;
        if ((e = event(&done)) != cudaSuccess || (e = cudaEventRecord(done, stream)) != cudaSuccess) break;
        for (int i : part) {
            dg_ctx *c = ctxs[i];
            if ((e = cudaStreamWaitEvent(c->stream, done, 0)) != cudaSuccess) break;
            CdftBatch a{};
            cdft_args(c, runs[(size_t)i], rd, a);
            if ((st = cdft_combine(c, runs[(size_t)i], a, rd)) != DG_OK) break;
        }
    }
    for (int i = 0; i < n && st == DG_OK && e == cudaSuccess; ++i) st = cdft_finish(ctxs[i], runs[(size_t)i]);
    for (auto &x : evs) cudaEventDestroy(x);
    if (st != DG_OK) return st;
    if (e != cudaSuccess) return fail(c0, DG_ECUDA, "shared contraction rounds: %s", cudaGetErrorString(e));
    return DG_OK;
}

static dg_status capture_steps(dg_ctx *const *ctxs, int n, void *const *costs, double spacing_m, const int *half,
                               cudaStream_t stream, cudaGraphExec_t *exec, int64_t *launches,
                               const TcRounds *rounds = nullptr)
{
    dg_ctx *c0 = ctxs[0];
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join((size_t)n, nullptr);
    CK(c0, cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    for (auto &e : join) CK(c0, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    std::vector<int> timing((size_t)n);
    std::vector<int64_t> l0((size_t)n);
    dg_status st = DG_OK;
    int64_t shared = 0;
    cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(fork, stream);
    for (int i = 0; i < n; ++i) {
        timing[i] = ctxs[i]->opt.timing;
        ctxs[i]->opt.timing = 0;
        l0[i] = ctxs[i]->launches;
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctxs[i]->stream, fork, 0);
    }
    if (rounds && e == cudaSuccess) st = shared_surfaces(ctxs, n, costs, *rounds, stream, &shared);
    for (int i = 0; i < n && e == cudaSuccess && st == DG_OK; ++i) {
        dg_ctx *c = ctxs[i];
        st = rounds ? step_device_post(c, costs[i], spacing_m, half[i]) : step_device(c, costs[i], spacing_m, half[i]);
        if (st == DG_OK) e = cudaEventRecord(join[i], c->stream);
        if (e == cudaSuccess && st == DG_OK) e = cudaStreamWaitEvent(stream, join[i], 0);
    }
    for (int i = 0; i < n; ++i) ctxs[i]->opt.timing = timing[i];
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(stream, &g);
    if (e == cudaSuccess) e = e2;
    int64_t total = shared;
    for (int i = 0; i < n; ++i) {
        const int64_t d = ctxs[i]->launches - l0[i];
        total += d;
        ctxs[i]->launches = l0[i];  // counted again at each replay
    }
    if (st == DG_OK && e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaEventDestroy(fork);
    for (auto &j : join) cudaEventDestroy(j);
    if (st != DG_OK) return st;
    if (e != cudaSuccess) return fail(c0, DG_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    *launches = total;
    return DG_OK;
}

dg_status dg_graph_capture(dg_ctx *c, void *cost, double spacing_m, double window_m)
{
    if (!c) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    c->err.clear();
    if (!cost) return fail(c, DG_EINVAL, "cost is NULL");
    if (!c->stream || c->stream == cudaStreamLegacy || c->stream == cudaStreamPerThread)
        return fail(c, DG_EUNSUPPORTED, "graph capture needs a context created on a non-default stream");
    int half = 0;
    dg_status st = refine_half(c, spacing_m, window_m, &half);
    if (st != DG_OK) return st;
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    // one uncaptured step allocates and plans everything; then the capture
    if ((st = prepare_step(c, half)) != DG_OK) return st;
    if ((st = step_device(c, cost, spacing_m, half)) != DG_OK) return st;
    dg_fix f;
    if ((st = read_fix(c, &f)) != DG_OK) return st;
    dg_ctx *const cs[1] = {c};
    void *const costs[1] = {cost};
    if ((st = capture_steps(cs, 1, costs, spacing_m, &half, c->stream, &c->graph, &c->graph_launches)) != DG_OK)
        return st;
    c->graph_gen = c->steps_gen;
    return DG_OK;
}

dg_status dg_graph_launch(dg_ctx *c)
{
    if (!c) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    c->err.clear();
    if (!c->graph) return fail(c, DG_ESTATE, "no graph has been captured");
    if (c->graph_gen != c->steps_gen || c->steps_dirty)
        return fail(c, DG_ESTATE, "a capture changed format, length or buffer since the graph was captured");
    CK(c, cudaGraphLaunch(c->graph, c->stream));
    c->launches += c->graph_launches;
    return DG_OK;
}

dg_status dg_graph_fix(dg_ctx *c, dg_fix *out)
{
    if (!c) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    c->err.clear();
    if (!out) return fail(c, DG_EINVAL, "out is NULL");
    if (!c->fix_host) return fail(c, DG_ESTATE, "no step has run");
    return read_fix(c, out);
}

}  // extern "C" (reopened below)

struct dg_batch {
    std::vector<dg_ctx *> ctxs;
    std::vector<uint64_t> gens;
    std::vector<cudaEvent_t> ready;  // work queued on each context's stream
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    int64_t launches = 0;
    std::string err;
    TcRounds rounds;       // shared contraction rounds (none: per-context launches)
    bool shared = false;
};

extern "C" {

dg_status dg_batch_capture(dg_ctx *const *ctxs, int32_t n, void *const *costs, double spacing_m, double window_m,
                           void *stream, dg_batch **out)
{
    if (!out) return fail(nullptr, DG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!ctxs || !costs || n < 1) return fail(nullptr, DG_EINVAL, "ctxs and costs must hold n >= 1 entries");
    cudaStream_t s = (cudaStream_t)stream;
    if (!s || s == cudaStreamLegacy || s == cudaStreamPerThread)
        return fail(nullptr, DG_EUNSUPPORTED, "graph capture needs a non-default stream");
    std::vector<int> half((size_t)n);
    for (int i = 0; i < n; ++i) {
        dg_ctx *c = ctxs[i];
        if (!c || !costs[i]) return fail(nullptr, DG_EINVAL, "context or cost %d is NULL", i);
        if (c->device != ctxs[0]->device) return fail(nullptr, DG_EINVAL, "the contexts must share one device");
        if (!c->stream || c->stream == cudaStreamLegacy || c->stream == cudaStreamPerThread)
            return fail(nullptr, DG_EUNSUPPORTED, "context %d is on a default stream", i);
        c->err.clear();
        dg_status st = refine_half(c, spacing_m, window_m, &half[i]);
        if (st == DG_OK) st = prepare_step(c, half[i]);
        if (st == DG_OK) st = step_device(c, costs[i], spacing_m, half[i]);
        dg_fix f;
        if (st == DG_OK) st = read_fix(c, &f);
        if (st != DG_OK) return fail(nullptr, st, "context %d: %s", i, c->err.c_str());
    }
    dg_batch *b = new (std::nothrow) dg_batch();
    if (!b) return fail(nullptr, DG_ENOMEM, "host allocation failed");
    b->ctxs.assign(ctxs, ctxs + n);
    for (int i = 0; i < n; ++i) b->gens.push_back(ctxs[i]->steps_gen);
    b->ready.assign((size_t)n, nullptr);
    for (auto &e : b->ready)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            for (auto &x : b->ready)
                if (x) cudaEventDestroy(x);
            delete b;
            return fail(nullptr, DG_ECUDA, "event creation failed");
        }
    b->stream = s;
    dg_status st = tc_rounds(ctxs, n, b->rounds, b->shared);
    if (st == DG_OK)
        st = capture_steps(ctxs, n, costs, spacing_m, half.data(), s, &b->graph, &b->launches,
                           b->shared ? &b->rounds : nullptr);
    if (st != DG_OK) {
        const std::string m = ctxs[0]->err;
        for (auto &e : b->ready) cudaEventDestroy(e);
        tc_rounds_free(b->rounds);
        delete b;
        return fail(nullptr, st, "%s", m.c_str());
    }
    *out = b;
    return DG_OK;
}

dg_status dg_batch_launch(dg_batch *b)
{
    if (!b || !b->graph) return fail(nullptr, DG_EINVAL, "no batch graph");
    for (size_t i = 0; i < b->ctxs.size(); ++i)
        if (b->ctxs[i]->steps_gen != b->gens[i] || b->ctxs[i]->steps_dirty)
            return fail(nullptr, DG_ESTATE, "context %zu changed a capture's format, length or buffer", i);
    // the steps read what was queued on the contexts' own streams (capture
    // loads): order the launch after it
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
        cudaError_t e = cudaEventRecord(b->ready[i], b->ctxs[i]->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ready[i], 0);
        if (e != cudaSuccess) return fail(nullptr, DG_ECUDA, "ordering the launch: %s", cudaGetErrorString(e));
    }
    const cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
    if (e != cudaSuccess) return fail(nullptr, DG_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
    return DG_OK;
}

dg_status dg_batch_fixes(dg_batch *b, dg_fix *out)
{
    if (!b || !out) return fail(nullptr, DG_EINVAL, "batch and out must not be NULL");
    const cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return fail(nullptr, DG_ECUDA, "cudaStreamSynchronize: %s", cudaGetErrorString(e));
    dg_status worst = DG_OK;
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
        dg_status st = read_fix(b->ctxs[i], &out[i]);
        if (st != DG_OK) {
            std::memset(&out[i], 0, sizeof(dg_fix));
            out[i].index = -1;
            if (worst == DG_OK) {
                worst = st;
                fail(nullptr, st, "context %zu: %s", i, b->ctxs[i]->err.c_str());
            }
        }
    }
    return worst;
}

int64_t dg_batch_launch_count(const dg_batch *b) { return b ? b->launches : -1; }

dg_status dg_batch_destroy(dg_batch *b)
{
    if (!b) return DG_OK;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (auto &e : b->ready)
        if (e) cudaEventDestroy(e);
    tc_rounds_free(b->rounds);
    delete b;
    return DG_OK;
}

int32_t dg_batch_rounds(const dg_batch *b) { return b && b->shared ? (int32_t)b->rounds.ctx.size() : 0; }

// ---------------------------------------------------------------------------
// Autotuning of the CDFT launch shape
// ---------------------------------------------------------------------------
namespace {
std::mutex g_tune_mutex;
// a tuned shape: chunk and tiles (CDFT) or rows (DIRECT)
struct TuneShape {
    int chunk = 0, tiles = 0, rows = 0;
};
std::map<std::string, TuneShape> g_tune_cache;

std::string tune_key(const dg_ctx *c)
{
    std::string k = std::to_string(c->G) + "/" + std::to_string(c->gd.nlon) + "/" + std::to_string(c->K) + "/" +
                    std::to_string(c->opt.algo) + "/" + std::to_string(c->opt.prec) + "/" +
                    std::to_string(c->opt.delay) + "/" + std::to_string(c->opt.contract) + "/" +
                    std::to_string(c->opt.acc) + "/" + std::to_string(c->fs);
    for (const auto &st : c->steps) k += "/" + std::to_string(st.n) + ":" + std::to_string(st.fmt);
    return k;
}
}  // namespace

dg_status dg_autotune(dg_ctx *c, void *cost, int32_t reps, dg_tuning *out)
{
    if (!c) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    c->err.clear();
    if (!cost || !out) return fail(c, DG_EINVAL, "cost and out must not be NULL");
    if (reps < 1 || reps > 100) return fail(c, DG_EINVAL, "reps must be in [1, 100]");
    for (int k = 0; k < c->K; ++k)
        if (!c->steps[k].loaded) return fail(c, DG_ESTATE, "snapshot %d has not been loaded", k);
    std::memset(out, 0, sizeof *out);
    const bool cdft = c->opt.algo == DG_ALGO_CDFT;
    auto apply = [&](const TuneShape &t) {
        if (cdft) {
            c->opt.chunk = t.chunk;
            c->opt.tiles = t.tiles;
            out->chunk = t.chunk;
            out->tiles = t.tiles;
        } else {
            c->opt.rows = t.rows;
            out->rows = t.rows;
        }
    };
    const std::string key = tune_key(c);
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            apply(it->second);
            out->cached = 1;
            return DG_OK;
        }
    }
    std::vector<TuneShape> shapes;
    if (cdft) {
        // admissible chunks: the automatic rule's bound on the estimated spacing
        std::vector<double> &span = c->cd.main_span;
        if (span.size() != (size_t)c->K || c->cd.main_lags.size() != (size_t)c->K)
            fdoa_spans(c, c->gd, span, &c->cd.main_lags);
        double dmax = 0.0;
        int64_t nmin = INT64_MAX;
        for (int k = 0; k < c->K; ++k) {
            dmax = std::max(dmax, span[k] * (1.0 + 1e-5) / kCdftBinSpan);
            nmin = std::min<int64_t>(nmin, c->steps[k].n);
        }
        const bool tc = c->opt.contract != DG_CONTRACT_FP32;
        std::vector<int> chunks;
        for (int m = 256; m <= (tc ? kCdftAutoMaxChunkTc : kCdftAutoMaxChunk); m *= 2)
            if (1.1 * m * dmax <= kCdftMDelta && (m <= kCdftAutoMaxChunk || m <= nmin)) chunks.push_back(m);
        if (chunks.empty()) chunks.push_back(auto_chunk(c, span, c->cd.main_lags, 0, c->K, tc));
        std::vector<int> tiles = {DG_TILES_ROWS};
        if (tc) {
            tiles.push_back(DG_TILES_LAGS);
            tiles.push_back(DG_TILES_HANKEL);
        }
        for (int m : chunks)
            for (int t : tiles) {
                if (t == DG_TILES_HANKEL && m > kLagTileMaxChunk) continue;
                if (t == DG_TILES_LAGS && m > kLagTileMaxChunk && m % kLagTileMaxChunk != 0) continue;
                TuneShape sh;
                sh.chunk = m;
                sh.tiles = t;
                shapes.push_back(sh);
            }
    } else {
        // grid rows per thread: candidates per CTA and the CTA's lag span
        // (16 rows of 4-tap interpolation weights spill registers: not tried)
        const std::vector<int> rows = c->opt.prec == DG_PREC_FP64         ? std::vector<int>{2, 4}
                                      : c->opt.delay == DG_DELAY_INTEGER ? std::vector<int>{4, 8, 16}
                                                                         : std::vector<int>{4, 8};
        for (int r : rows) {
            TuneShape sh;
            sh.rows = r;
            shapes.push_back(sh);
        }
    }
    const dg_options saved = c->opt;
    const size_t esz = c->opt.prec == DG_PREC_FP64 ? 8 : 4;
    dg_status st = ensure(c, &c->surf, &c->surf_bytes, esz * (size_t)c->G * c->K);
    if (st != DG_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    double best = 1e300;
    TuneShape best_sh = shapes[0];
    c->opt.timing = 0;  // restored with the saved options
    for (const TuneShape &sh : shapes) {
        if (cdft) {
            c->opt.chunk = sh.chunk;
            c->opt.tiles = sh.tiles;
        } else {
            c->opt.rows = sh.rows;
        }
        std::vector<float> ms;
        for (int r = 0; r <= reps && st == DG_OK; ++r) {
            if (r > 0 && cudaEventRecord(e0, c->stream) != cudaSuccess) st = DG_ECUDA;
            if (st == DG_OK) st = run_surface(c, c->gd, c->xyz, c->G, c->surf, cost, false);
            if (st == DG_OK && r > 0 && cudaEventRecord(e1, c->stream) != cudaSuccess) st = DG_ECUDA;
            if (st == DG_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) st = DG_ECUDA;
            if (st == DG_OK) st = check_latched(c);
            float x = 0.f;
            if (st == DG_OK && r > 0) {
                cudaEventElapsedTime(&x, e0, e1);
                ms.push_back(x);
            }
        }
        if (st != DG_OK) break;
        std::sort(ms.begin(), ms.end());
        const double med = ms[ms.size() / 2];
        ++out->tried;
        if (med < best) {
            best = med;
            best_sh = sh;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->opt = saved;
    if (st != DG_OK) {
        if (c->err.empty()) fail(c, st, "a timed surface failed");
        return st;
    }
    apply(best_sh);
    out->ms = best;
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    g_tune_cache[key] = best_sh;
    return DG_OK;
}

dg_status dg_grid_ecef(dg_ctx *c, double *xyz_out)
{
    if (!c) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    c->err.clear();
    if (!xyz_out) return fail(c, DG_EINVAL, "xyz_out is NULL");
    CK(c, cudaMemcpyAsync(xyz_out, c->xyz, sizeof(double) * 3 * (size_t)c->G, cudaMemcpyDeviceToDevice,
                          c->stream));
    return DG_OK;
}

dg_status dg_step_geometry(dg_ctx *c, int32_t step, int32_t *lag, double *D, double *nu)
{
    if (!c) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    c->err.clear();
    if (step < 0 || step >= c->K) return fail(c, DG_EINVAL, "step %d outside [0, %d)", step, c->K);
    {
        Timed t(c, DG_K_GRID);
        CK(c, launch_step_geometry(c->gd, c->xyz, c->eph + 12 * (size_t)step, c->fs, c->lambda,
                                   c->opt.delay, lag, D, nu, c->stream));
        t.done(1);
    }
    return DG_OK;
}

dg_status dg_kernel_time(dg_ctx *c, int32_t cls, double *ms, int64_t *launches)
{
    if (!c) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    c->err.clear();
    if (cls < 0 || cls >= DG_K_NCLASS) return fail(c, DG_EINVAL, "unknown kernel class %d", cls);
    CK(c, cudaStreamSynchronize(c->stream));
    for (auto &t : c->pending) {
        float v = 0;
        cudaEventElapsedTime(&v, t.a, t.b);
        c->ms[t.cls] += v;
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    c->pending.clear();
    if (ms) *ms = c->ms[cls];
    if (launches) *launches = c->nl[cls];
    return DG_OK;
}

dg_status dg_reset_counters(dg_ctx *c)
{
    if (!c) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    c->err.clear();
    CK(c, cudaStreamSynchronize(c->stream));
    for (auto &t : c->pending) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    c->pending.clear();
    for (int i = 0; i < DG_K_NCLASS; ++i) {
        c->ms[i] = 0;
        c->nl[i] = 0;
    }
    c->launches = 0;
    return DG_OK;
}

int64_t dg_launch_count(const dg_ctx *c) { return c ? c->launches : -1; }

dg_status dg_cdft_chunks(const dg_ctx *c, int32_t *min_chunk, int32_t *max_chunk)
{
    if (!c) return DG_EINVAL;
    const bool any = c->cd_chunk_max > 0;
    if (min_chunk) *min_chunk = any ? c->cd_chunk_min : 0;
    if (max_chunk) *max_chunk = any ? c->cd_chunk_max : 0;
    return DG_OK;
}

dg_status dg_cdft_work(const dg_ctx *c, int64_t *bucket_chunks, int64_t *candidate_chunks)
{
    if (!c) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    unsigned long long w[2] = {0, 0};
    if (c->cd.work) {  // counted on the device by the plan: wait for the stream
        if (cudaMemcpyAsync(w, c->cd.work, sizeof w, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return fail(nullptr, DG_ECUDA, "reading the CDFT work counters failed");
    }
    if (bucket_chunks) *bucket_chunks = (int64_t)w[0];
    if (candidate_chunks) *candidate_chunks = (int64_t)w[1];
    return DG_OK;
}

dg_status dg_destroy(dg_ctx *c)
{
    if (!c) return DG_OK;
    cudaStream_t s = c->stream;
    for (auto &t : c->pending) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    auto fr = [&](void *p) {
        if (p) cudaFreeAsync(p, s);
    };
    fr(c->xyz);
    fr(c->eph);
    fr(c->steps_d);
    fr(c->surf);
    fr(c->amax_tmp);
    fr(c->amax_res);
    fr(c->amax_fine);
    fr(c->fix_dev);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    fr(c->err_d);
    fr(c->det_count);
    fr(c->det_cand);
    fr(c->det_out);
    fr(c->loc.xyz);
    fr(c->loc.surf);
    fr(c->loc.cost);
    fr(c->cd.lr);
    fr(c->reg_res);
    fr(c->co.lag);
    fr(c->co.nu);
    fr(c->co.lmm);
    fr(c->co.nmm);
    fr(c->co.st);
    fr(c->co.P);
    fr(c->co.A);
    fr(c->co.part);
    fr(c->cd.main_layout.bbase);
    fr(c->cd.main_layout.gbase);
    fr(c->cd.loc_layout.bbase);
    fr(c->cd.loc_layout.gbase);
    fr(c->cd.layout);
    fr(c->cd.Mcs);
    fr(c->cd.work);
    fr(c->cd.candL);
    fr(c->cd.order);
    fr(c->cd.nuS);
    fr(c->cd.g2b);
    fr(c->cd.candNu);
    fr(c->cd.candMu);
    fr(c->cd.muS);
    fr(c->cd.need);
    fr(c->cd.xyzf);
    fr(c->cd.ephf);
    fr(c->cd.count);
    fr(c->cd.offs);
    fr(c->cd.subcnt);
    fr(c->cd.nur);
    fr(c->cd.nubase);
    fr(c->cd.delta);
    fr(c->cd.V);
    fr(c->cd.W);
    fr(c->cd.tbase);
    fr(c->cd.hbase);
    fr(c->cd.btab);
    for (auto &st : c->steps) {
        fr(st.y1);
        fr(st.y2);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (c->amax_host) cudaFreeHost(c->amax_host);
    if (c->reg_host) cudaFreeHost(c->reg_host);
    if (c->fix_host) cudaFreeHost(c->fix_host);
    if (c->err_h) cudaFreeHost(c->err_h);
    delete c;
    if (e != cudaSuccess) return fail(nullptr, DG_ECUDA, "dg_destroy: %s", cudaGetErrorString(e));
    return DG_OK;
}

// ---------------------------------------------------------------------------
// Coarse delay-Doppler maps back-projected onto the grid's cells.
// ---------------------------------------------------------------------------
dg_status dg_coarse_maps(dg_ctx *c, int32_t bins, int32_t chunk, float *maps)
{
    if (!c) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    c->err.clear();
    if (!maps) return fail(c, DG_EINVAL, "maps is NULL");
    if (c->gd.row0 != 0 || c->gd.nrows != c->gd.nlat)
        return fail(c, DG_EUNSUPPORTED, "dg_coarse_maps needs a context over the whole grid (no row shard)");
    if (c->gd.nlat < 2 || c->gd.nlon < 2) return fail(c, DG_EINVAL, "dg_coarse_maps needs at least 2 x 2 nodes");
    if (bins != 0 && (bins < 2 || bins > 256)) return fail(c, DG_EINVAL, "bins %d outside 2..256 (0: auto)", bins);
    if (chunk != 0 && (chunk < 1 || chunk > 4096 || (chunk & (chunk - 1))))
        return fail(c, DG_EINVAL, "chunk %d is not a power of two in 1..4096 (0: auto)", chunk);
    int nmax = 0;
    for (int k = 0; k < c->K; ++k) {
        if (!c->steps[k].loaded) return fail(c, DG_ESTATE, "snapshot %d has not been loaded", k);
        nmax = std::max(nmax, (int)c->steps[k].n);
    }
    // planning from the host's lattice estimate of the FDOA span (25 % margin)
    std::vector<double> &spans = c->cd.main_span;  // cached until the grid changes
    if (spans.size() != (size_t)c->K) fdoa_spans(c, c->gd, spans);
    double span = 0.0;
    for (int k = 0; k < c->K; ++k) span = std::max(span, spans[k]);
    span *= 1.25;
    int M = chunk;
    if (M == 0) {  // the chunk's phase error (nu_q - nu_c) m stays below 1/8 cycle
        M = 1024;
        while (M > 1 && 0.5 * span * M > 0.125) M >>= 1;
    }
    int Q = bins;
    if (Q == 0) {  // two bins per Doppler resolution cell 1 / N
        Q = (int)std::ceil(2.0 * nmax * span) + 1;
        Q = std::min(256, std::max(16, (Q + 7) / 8 * 8));
    }
    const int nb_max = (nmax + M - 1) / M;
    if (nb_max > 65535) return fail(c, DG_EUNSUPPORTED, "chunk %d leaves %d chunks (at most 65535)", M, nb_max);
    const double diam = grid_diameter(c->gd);
    int nlag_cap = 0;
    for (int k = 0; k < c->K; ++k) nlag_cap = std::max(nlag_cap, lag_slots(c->eph_host[k], c->fs, diam));
    const size_t KG = (size_t)c->K * (size_t)c->G, K = (size_t)c->K;
    CoarseBufs &b = c->co;
    dg_status st;
    if ((st = ensure(c, (void **)&b.lag, &b.lag_cap, sizeof(int) * KG)) != DG_OK) return st;
    if ((st = ensure(c, (void **)&b.nu, &b.nu_cap, sizeof(float) * KG)) != DG_OK) return st;
    if ((st = ensure(c, (void **)&b.lmm, &b.lmm_cap, sizeof(int) * 2 * K)) != DG_OK) return st;
    if ((st = ensure(c, (void **)&b.nmm, &b.nmm_cap, sizeof(unsigned long long) * 2 * K)) != DG_OK) return st;
    if ((st = ensure(c, (void **)&b.st, &b.st_cap, sizeof(CoarseStep) * K)) != DG_OK) return st;
    if ((st = ensure(c, (void **)&b.P, &b.P_cap, sizeof(float2) * K * nb_max * (size_t)nlag_cap)) != DG_OK) return st;
    if ((st = ensure(c, (void **)&b.A, &b.A_cap, sizeof(float) * K * (size_t)nlag_cap * Q)) != DG_OK) return st;
    if ((st = ensure(c, (void **)&b.part, &b.part_cap, sizeof(double) * K * coarse_bin_tiles(nlag_cap))) != DG_OK)
        return st;
    if ((st = push_steps(c)) != DG_OK) return st;
    if ((st = ensure_ephf(c)) != DG_OK) return st;
    if (c->cd.xyzf_cap < (size_t)c->G) {
        if ((st = grow(c, &c->cd.xyzf, 6 * (size_t)c->G)) != DG_OK) return st;
        c->cd.xyzf_cap = (size_t)c->G;
    }
    CoarseArgs a{};
    a.xyz = c->xyz;
    a.xyzf = c->cd.xyzf;
    a.ephf = c->cd.ephf;
    a.fsc_hi = (float)(c->fs / kC);
    a.fsc_lo = (float)(c->fs / kC - (double)a.fsc_hi);
    a.ilf_hi = (float)(1.0 / (c->lambda * c->fs));
    a.ilf_lo = (float)(1.0 / (c->lambda * c->fs) - (double)a.ilf_hi);
    a.G = c->G;
    a.nlat = c->gd.nlat;
    a.nlon = c->gd.nlon;
    a.eph = c->eph;
    a.steps = c->steps_d;
    a.K = c->K;
    a.fs = c->fs;
    a.lambda = c->lambda;
    a.Q = Q;
    a.M = M;
    a.nlag_cap = nlag_cap;
    a.nb_max = nb_max;
    a.lag = b.lag;
    a.nu = b.nu;
    a.lmm = b.lmm;
    a.nmm = b.nmm;
    a.st = b.st;
    a.P = b.P;
    a.A = b.A;
    a.part = b.part;
    a.maps = maps;
    a.err = c->err_d;
    {
        Timed t(c, DG_K_COARSE);
        int n = 1;
        CK(c, launch_ecef_split(c->xyz, c->G, c->cd.xyzf, c->stream));
        CK(c, launch_coarse(a, c->stream, &n));
        t.done(n);
    }
    CK(c, cudaMemcpyAsync(c->err_h, c->err_d, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    b.Q = Q;
    b.M = M;
    b.nlag_cap = nlag_cap;
    b.nb_max = nb_max;
    return DG_OK;
}

dg_status dg_coarse_inspect(dg_ctx *c, float *caf, dg_coarse_step *steps, int32_t *shape)
{
    if (!c) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    c->err.clear();
    const CoarseBufs &b = c->co;
    if (b.Q == 0) return fail(c, DG_ESTATE, "no coarse maps have been computed on this context");
    if (shape) {
        shape[0] = b.Q;
        shape[1] = b.M;
        shape[2] = b.nlag_cap;
    }
    if (caf)
        CK(c, cudaMemcpyAsync(caf, b.A, sizeof(float) * (size_t)c->K * b.nlag_cap * b.Q, cudaMemcpyDeviceToDevice,
                              c->stream));
    if (steps) {
        std::vector<CoarseStep> h(c->K);
        CK(c, cudaMemcpyAsync(h.data(), b.st, sizeof(CoarseStep) * c->K, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        for (int k = 0; k < c->K; ++k) {
            steps[k].l0 = h[k].l0;
            steps[k].nlag = h[k].nlag;
            steps[k].nu_lo = h[k].nu_lo;
            steps[k].delta = h[k].delta;
            steps[k].nu_c = h[k].nu_c;
            steps[k].mu = h[k].mu;
        }
        return check_latched(c);
    }
    return DG_OK;
}

// ---------------------------------------------------------------------------
// Search of several regions with one host synchronisation.
// ---------------------------------------------------------------------------
dg_status dg_search_regions(dg_ctx *c, const dg_grid *regions, int32_t n, void *costs, double spacing_m,
                            double window_m, dg_fix *out, int32_t *best)
{
    if (!c) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    c->err.clear();
    if (!regions || !costs || !out) return fail(c, DG_EINVAL, "regions, costs and out must not be NULL");
    if (n < 1 || n > 256) return fail(c, DG_EINVAL, "n = %d outside 1..256", n);
    for (int r = 0; r < n; ++r) {
        dg_status st = validate_grid(c, &regions[r]);
        if (st != DG_OK) return st;
        if (regions[r].nlat != regions[0].nlat || regions[r].nlon != regions[0].nlon)
            return fail(c, DG_EINVAL, "regions must all have the same number of nodes");
    }
    for (int k = 0; k < c->K; ++k)
        if (!c->steps[k].loaded) return fail(c, DG_ESTATE, "snapshot %d has not been loaded", k);
    const int64_t G = (int64_t)regions[0].nlat * regions[0].nlon;
    const size_t esz = c->opt.prec == DG_PREC_FP64 ? 8 : 4;
    if (c->reg_cap < (size_t)n) {
        if (c->reg_res) CK(c, cudaFreeAsync(c->reg_res, c->stream));
        c->reg_res = nullptr;
        if (c->reg_host) {
            CK(c, cudaStreamSynchronize(c->stream));
            cudaFreeHost(c->reg_host);
            c->reg_host = nullptr;
        }
        c->reg_cap = 0;
        CK(c, cudaMallocAsync((void **)&c->reg_res, sizeof(ArgmaxResult) * n, c->stream));
        CK(c, cudaMallocHost((void **)&c->reg_host, sizeof(ArgmaxResult) * n));
        c->reg_cap = (size_t)n;
    }
    dg_status st;
    for (int r = 0; r < n; ++r) {
        if ((st = dg_set_grid(c, &regions[r])) != DG_OK) return st;
        if ((st = ensure(c, &c->surf, &c->surf_bytes, esz * (size_t)G * c->K)) != DG_OK) return st;
        if ((st = ensure(c, &c->amax_tmp, &c->amax_tmp_bytes, argmax_tmp_bytes(G))) != DG_OK) return st;
        void *cr = (char *)costs + esz * (size_t)G * r;
        if ((st = run_surface(c, c->gd, c->xyz, G, c->surf, cr, false)) != DG_OK) return st;
        int nl = 0;
        {
            Timed t(c, DG_K_ARGMAX);
            CK(c, launch_argmax(cr, G, c->opt.prec, c->gd, c->amax_tmp, c->reg_res + r, &nl, c->stream));
            t.done(nl);
        }
    }
    CK(c, cudaMemcpyAsync(c->reg_host, c->reg_res, sizeof(ArgmaxResult) * n, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if ((st = check_latched(c)) != DG_OK) return st;
    int b = -1;
    for (int r = 0; r < n; ++r)
        if (c->reg_host[r].idx >= 0 && (b < 0 || c->reg_host[r].val > c->reg_host[b].val)) b = r;
    if (b < 0) return fail(c, DG_EINVAL, "no region holds a finite value");
    if ((st = dg_set_grid(c, &regions[b])) != DG_OK) return st;
    if ((st = dg_argmax_refine(c, (char *)costs + esz * (size_t)G * b, spacing_m, window_m, out)) != DG_OK) return st;
    if (best) *best = b;
    return DG_OK;
}

}  // extern "C"

extern "C" dg_status dg_debug_tc_wait_limit(uint32_t polls)
{
    g_tc_wait_polls.store(polls, std::memory_order_relaxed);
    return DG_OK;
}
