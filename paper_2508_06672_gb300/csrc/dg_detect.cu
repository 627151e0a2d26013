// dg_detect.cu -- threshold detection of emitters on an accumulated surface
// (Algorithm 1, last step). A node is a peak when its value is >= the
// threshold and it is the maximum of the (2r+1) x (2r+1) window around it;
// among equal values the lowest linear index wins (one peak per plateau).
// Peaks are sorted by value (descending), ties by index, in one CTA.
#include <cfloat>

#include "dg_internal.cuh"

namespace dg {

template <typename T>
__global__ void __launch_bounds__(256) k_detect_mark(const T *__restrict__ v, int nrows, int nlon, double thr, int r,
                                                     int cap, int *count, int64_t *cand)
{
    const int64_t G = (int64_t)nrows * nlon;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < G; p += (int64_t)gridDim.x * blockDim.x) {
        const T x = v[p];
        if (!((double)x >= thr)) continue;
        const int i = (int)(p / nlon), j = (int)(p % nlon);
        bool peak = true;
        for (int di = -r; di <= r && peak; ++di) {
            const int ii = i + di;
            if (ii < 0 || ii >= nrows) continue;
            for (int dj = -r; dj <= r; ++dj) {
                const int jj = j + dj;
                if ((di == 0 && dj == 0) || jj < 0 || jj >= nlon) continue;
                const int64_t q = (int64_t)ii * nlon + jj;
                const T y = v[q];
                if (y > x || (y == x && q < p)) {
                    peak = false;
                    break;
                }
            }
        }
        if (peak) {
            const int k = atomicAdd(count, 1);
            if (k < cap) cand[k] = p;
        }
    }
}

// One CTA: bitonic sort of min(count, cap) candidates (cap a power of two <=
// kDetectCap) by (value desc, index asc); the first max_peaks become peak records.
template <typename T>
__global__ void __launch_bounds__(1024) k_detect_sort(const T *__restrict__ v, const int *count, const int64_t *cand,
                                                      int cap, int max_peaks, GridDev g, DetectPeak *out)
{
    __shared__ double sv[kDetectCap];
    __shared__ int64_t si[kDetectCap];
    const int n = min(*count, cap);
    for (int t = threadIdx.x; t < cap; t += blockDim.x) {
        if (t < n) {
            si[t] = cand[t];
            sv[t] = (double)v[cand[t]];
        } else {
            si[t] = INT64_MAX;
            sv[t] = -DBL_MAX;
        }
    }
    __syncthreads();
    for (int k = 2; k <= cap; k <<= 1)
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int t = threadIdx.x; t < cap; t += blockDim.x) {
                const int u = t ^ jj;
                if (u > t) {
                    // "a before b": larger value, or equal value and lower index
                    const bool t_first = sv[t] > sv[u] || (sv[t] == sv[u] && si[t] < si[u]);
                    const bool up = (t & k) == 0;
                    if (up != t_first) {
                        const double tv = sv[t];
                        sv[t] = sv[u];
                        sv[u] = tv;
                        const int64_t ti = si[t];
                        si[t] = si[u];
                        si[u] = ti;
                    }
                }
            }
            __syncthreads();
        }
    const GridStep st = grid_step(g);
    for (int t = threadIdx.x; t < min(n, max_peaks); t += blockDim.x) {
        const int i = g.row0 + (int)(si[t] / g.nlon), j = (int)(si[t] % g.nlon);
        double lat, lon;
        grid_node(g, st, i, j, lat, lon);
        out[t].index = si[t];
        out[t].i = i;
        out[t].j = j;
        out[t].lat_rad = lat;
        out[t].lon_rad = lon;
        out[t].value = sv[t];
    }
}

cudaError_t launch_detect(const void *v, int prec, const GridDev &g, double thr, int r, int cap, int max_peaks,
                          int *count, int64_t *cand, DetectPeak *out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    const int64_t G = (int64_t)g.nrows * g.nlon;
    int64_t blocks = (G + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    if (prec == DG_PREC_FP64) {
        k_detect_mark<double><<<(unsigned)blocks, 256, 0, s>>>((const double *)v, g.nrows, g.nlon, thr, r, cap, count, cand);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_detect_sort<double><<<1, 1024, 0, s>>>((const double *)v, count, cand, cap, max_peaks, g, out);
    } else {
        k_detect_mark<float><<<(unsigned)blocks, 256, 0, s>>>((const float *)v, g.nrows, g.nlon, thr, r, cap, count, cand);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_detect_sort<float><<<1, 1024, 0, s>>>((const float *)v, count, cand, cap, max_peaks, g, out);
    }
    return cudaGetLastError();
}

}  // namespace dg
