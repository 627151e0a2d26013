// dg_reduce.cu -- non-coherent accumulation over snapshots and the argmax
// (Algorithm 1: sum the position-domain correlation grids; Sec. III: the
// maximum of S is the maximum-likelihood estimate).
#include <cfloat>

#include "dg_internal.cuh"

namespace dg {

// out[p] = sum_{k=0}^{K-1} surf[k][p], always in that order (deterministic).
// Vectorised by 4 along p where G allows; HBM-bound (K reads + 1 write).
template <typename T>
__global__ void __launch_bounds__(256) k_accumulate(const T *__restrict__ surf, int K, int64_t G,
                                                    T *__restrict__ out)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < G;
         p += (int64_t)gridDim.x * blockDim.x) {
        T s = surf[p];
        for (int k = 1; k < K; ++k) s += __ldcs(surf + (int64_t)k * G + p);
        out[p] = s;
    }
}

cudaError_t launch_accumulate(const void *surf, int K, int64_t G, int prec, void *out, cudaStream_t s)
{
    int64_t blocks = (G + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    if (prec == DG_PREC_FP64)
        k_accumulate<double><<<(unsigned)blocks, 256, 0, s>>>((const double *)surf, K, G, (double *)out);
    else
        k_accumulate<float><<<(unsigned)blocks, 256, 0, s>>>((const float *)surf, K, G, (float *)out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// argmax: (value, index) pairs; a beats b if a is valid and (b is invalid, or
// a.val > b.val, or equal values and a.idx < b.idx). NaN is never valid.
// ---------------------------------------------------------------------------
struct VI {
    double val;
    int64_t idx;
};

__device__ __forceinline__ bool beats(const VI &a, const VI &b)
{
    if (a.idx < 0) return false;
    if (b.idx < 0) return true;
    return a.val > b.val || (a.val == b.val && a.idx < b.idx);
}

__device__ __forceinline__ VI warp_best(VI v)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        VI o;
        o.val = __shfl_xor_sync(0xffffffffu, v.val, d);
        o.idx = __shfl_xor_sync(0xffffffffu, v.idx, d);
        if (beats(o, v)) v = o;
    }
    return v;
}

__device__ __forceinline__ VI block_best(VI v)
{
    __shared__ VI sh[32];
    v = warp_best(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (warp == 0) {
        v = lane < nw ? sh[lane] : VI{0.0, -1};
        v = warp_best(v);
    }
    return v;  // valid in thread 0
}

template <typename T>
__global__ void __launch_bounds__(1024) k_argmax_partial(const T *__restrict__ v, int64_t n, VI *part)
{
    VI best{0.0, -1};
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double x = (double)v[p];
        if (x == x && (best.idx < 0 || x > best.val)) best = VI{x, p};  // p increases per thread
    }
    best = block_best(best);
    if (threadIdx.x == 0) part[blockIdx.x] = best;
}

// Offset (in nodes, within [-0.5, 0.5]) of the vertex of the parabola
// through the values at c - stride, c, c + stride: 0.5 (a - d) / (a - 2b + d)
// where that curvature is negative, 0 at an edge, on a flat or non-concave
// triple, or with a non-finite neighbour.
template <typename T>
__device__ __forceinline__ double parabola_offset(const T *v, int64_t c, int64_t stride, bool lo, bool hi)
{
    if (!lo || !hi) return 0.0;
    const double a = (double)v[c - stride], b = (double)v[c], d = (double)v[c + stride];
    const double den = __dadd_rn(__dsub_rn(a, __dmul_rn(2.0, b)), d);
    if (!(den < 0.0)) return 0.0;
    const double x = __ddiv_rn(__dmul_rn(0.5, __dsub_rn(a, d)), den);
    return x != x ? 0.0 : fmin(0.5, fmax(-0.5, x));
}

__global__ void __launch_bounds__(1024) k_argmax_final(const VI *part, int nparts, GridDev g,
                                                       ArgmaxResult *res, const ArgmaxResult *centre,
                                                       const void *v, int prec)
{
    if (centre) centre_on(g, centre);
    VI best{0.0, -1};
    for (int p = threadIdx.x; p < nparts; p += blockDim.x)
        if (beats(part[p], best)) best = part[p];
    best = block_best(best);
    if (threadIdx.x == 0) {
        res->val = best.val;
        res->idx = best.idx;
        res->lat_rad = 0.0;
        res->lon_rad = 0.0;
        res->sub_lat_rad = 0.0;
        res->sub_lon_rad = 0.0;
        if (best.idx >= 0) {
            const GridStep st = grid_step(g);
            const int il = (int)(best.idx / g.nlon), j = (int)(best.idx % g.nlon);
            double lat, lon;
            grid_node(g, st, g.row0 + il, j, lat, lon);
            res->lat_rad = lat;
            res->lon_rad = lon;
            // neighbours within the surface (the shard's rows, the grid's columns)
            double di, dj;
            if (prec == DG_PREC_FP64) {
                const double *d = (const double *)v;
                di = parabola_offset(d, best.idx, g.nlon, il > 0, il < g.nrows - 1);
                dj = parabola_offset(d, best.idx, 1, j > 0, j < g.nlon - 1);
            } else {
                const float *f = (const float *)v;
                di = parabola_offset(f, best.idx, g.nlon, il > 0, il < g.nrows - 1);
                dj = parabola_offset(f, best.idx, 1, j > 0, j < g.nlon - 1);
            }
            res->sub_lat_rad = __dadd_rn(lat, __dmul_rn(di, st.dlat));
            res->sub_lon_rad = __dadd_rn(lon, __dmul_rn(dj, st.dlon));
        }
    }
}

static int argmax_blocks(int64_t n)
{
    int64_t b = (n + 1023) / 1024;
    if (b > 152 * 2) b = 152 * 2;
    if (b < 1) b = 1;
    return (int)b;
}

size_t argmax_tmp_bytes(int64_t n) { return sizeof(VI) * (size_t)argmax_blocks(n); }

cudaError_t launch_argmax(const void *v, int64_t n, int prec, const GridDev &g, void *tmp,
                          ArgmaxResult *res, int *launches, cudaStream_t s, const ArgmaxResult *centre)
{
    const int nb = argmax_blocks(n);
    VI *part = reinterpret_cast<VI *>(tmp);
    if (prec == DG_PREC_FP64)
        k_argmax_partial<double><<<nb, 1024, 0, s>>>((const double *)v, n, part);
    else
        k_argmax_partial<float><<<nb, 1024, 0, s>>>((const float *)v, n, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_argmax_final<<<1, 1024, 0, s>>>(part, nb, g, res, centre, v, prec);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

// One thread: the fields of dg_fix as dg_argmax_refine fills them.
__global__ void k_make_fix(const ArgmaxResult *coarse, const ArgmaxResult *fine, GridDev g, int n, dg_fix *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    dg_fix f;
    memset(&f, 0, sizeof f);
    f.index = coarse->idx;
    if (coarse->idx >= 0) {
        f.i = g.row0 + (int)(coarse->idx / g.nlon);
        f.j = (int)(coarse->idx % g.nlon);
    }
    f.lat_deg = coarse->lat_rad * (180.0 / kPi);
    f.lon_deg = coarse->lon_rad * (180.0 / kPi);
    f.cost = coarse->val;
    f.sub_lat_deg = coarse->sub_lat_rad * (180.0 / kPi);
    f.sub_lon_deg = coarse->sub_lon_rad * (180.0 / kPi);
    if (fine && coarse->idx >= 0) {
        f.refine_n = n;
        f.ri = f.rj = -1;  // no finite value on the refinement grid
        if (fine->idx >= 0) {
            f.ri = (int)(fine->idx / n);
            f.rj = (int)(fine->idx % n);
        }
        f.refined_lat_deg = fine->lat_rad * (180.0 / kPi);
        f.refined_lon_deg = fine->lon_rad * (180.0 / kPi);
        f.refined_cost = fine->val;
        if (fine->idx >= 0) {
            f.sub_lat_deg = fine->sub_lat_rad * (180.0 / kPi);
            f.sub_lon_deg = fine->sub_lon_rad * (180.0 / kPi);
        }
    }
    *out = f;
}

cudaError_t launch_make_fix(const ArgmaxResult *coarse, const ArgmaxResult *fine, const GridDev &g, int n,
                            dg_fix *out, cudaStream_t s)
{
    k_make_fix<<<1, 32, 0, s>>>(coarse, fine, g, n, out);
    return cudaGetLastError();
}

}  // namespace dg
