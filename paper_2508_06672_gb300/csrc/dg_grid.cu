// dg_grid.cu -- candidate grid to ECEF (Algorithm 1, first step; Sec. III)
// and the per-snapshot geometry table used for inspection (Eq. 3-10).
#include "dg_internal.cuh"

namespace dg {

// One thread per node of the shard. Geodetic (lat, lon, h = 0) on WGS-84 to
// ECEF: N = a / sqrt(1 - e2 sin^2 lat), x = N cos lat cos lon,
// y = N cos lat sin lon, z = N (1 - e2) sin lat. Output SoA [3][G].
__global__ void __launch_bounds__(256) k_grid_ecef(GridDev g, double *__restrict__ xyz, const ArgmaxResult *centre)
{
    if (centre) centre_on(g, centre);
    const int64_t G = (int64_t)g.nrows * g.nlon;
    const GridStep st = grid_step(g);
    const double e2 = kF * (2.0 - kF);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < G;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = g.row0 + (int)(p / g.nlon);
        const int j = (int)(p % g.nlon);
        double lat, lon;
        grid_node(g, st, i, j, lat, lon);
        double sl, cl, so, co;
        sincos(lat, &sl, &cl);
        sincos(lon, &so, &co);
        const double n = __ddiv_rn(kA, __dsqrt_rn(__dsub_rn(1.0, __dmul_rn(__dmul_rn(e2, sl), sl))));
        xyz[p] = __dmul_rn(__dmul_rn(n, cl), co);
        xyz[G + p] = __dmul_rn(__dmul_rn(n, cl), so);
        xyz[2 * G + p] = __dmul_rn(__dmul_rn(n, 1.0 - e2), sl);
    }
}

cudaError_t launch_grid_ecef(const GridDev &g, double *xyz, cudaStream_t s, const ArgmaxResult *centre)
{
    const int64_t G = (int64_t)g.nrows * g.nlon;
    int64_t blocks = (G + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_grid_ecef<<<(unsigned)blocks, 256, 0, s>>>(g, xyz, centre);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_step_geometry(int64_t G, const double *__restrict__ xyz,
                                                       const double *__restrict__ eph_k, double fs,
                                                       double lambda, int delay_mode, int *lag,
                                                       double *Dout, double *nuout)
{
    double e[12];
#pragma unroll
    for (int t = 0; t < 12; ++t) e[t] = __ldg(eph_k + t);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < G;
         p += (int64_t)gridDim.x * blockDim.x) {
        double D, nu;
        geometry(xyz[p], xyz[G + p], xyz[2 * G + p], e, fs, lambda, D, nu);
        if (lag) lag[p] = lag_of(D, delay_mode);
        if (Dout) Dout[p] = D;
        if (nuout) nuout[p] = nu;
    }
}

cudaError_t launch_step_geometry(const GridDev &g, const double *xyz, const double *eph_k,
                                 double fs, double lambda, int delay_mode, int *lag, double *D,
                                 double *nu, cudaStream_t s)
{
    const int64_t G = (int64_t)g.nrows * g.nlon;
    int64_t blocks = (G + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_step_geometry<<<(unsigned)blocks, 256, 0, s>>>(G, xyz, eph_k, fs, lambda, delay_mode, lag, D, nu);
    return cudaGetLastError();
}

}  // namespace dg
