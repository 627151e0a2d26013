/*
 * dg_oracle.c -- plain FP64 CPU oracle for direct geolocation.
 *
 * TEST INFRASTRUCTURE. Only the tests, __graft_entry__.smoke() and the CPU
 * baseline / reference arm of bench.py may load this. The CUDA library never
 * calls it, and it shares no code, header, table or constant with the CUDA
 * library.
 *
 * It is the definition of Sec. III written out, with no blocking, fusion or
 * reordering: for every candidate and every snapshot, the geometry of
 * Eq. 3-8, the expected lag of Eq. 9 and FDOA of Eq. 10, the correlation of
 * Eq. 11 as a plain sum over samples, then the sum over snapshots of
 * Algorithm 1 and the argmax. Readings where the paper is silent:
 *   - Eq. 9 is read as round(dtau * fs) (the printed "/ fs" has wrong units);
 *     round() is half away from zero.
 *   - Samples outside [0, N) are zero (the sum runs over the overlap).
 *   - t_k = k / fs from the first sample of each snapshot (Sec. II, Eq. 2).
 *   - The exponent is evaluated as 2 pi frac(dfreq * k / fs).
 *   - The fractional-delay mode (not in the paper, which rounds) uses 4-tap
 *     cubic Lagrange interpolation at taps -1..2 around floor(D).
 *   - Accumulation is sum_k |C_k|^2 (power) or sum_k |C_k| (the paper's S).
 *   - Grid nodes are regular in latitude/longitude, centred on (lat0, lon0),
 *     with spacing given in metres at the centre latitude through the WGS-84
 *     meridian and prime-vertical radii; altitude 0 on the WGS-84 ellipsoid.
 * Every floating-point expression that feeds the integer lag is evaluated in
 * the order written here; build with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define DGO_C_LIGHT 299792458.0
#define DGO_WGS84_A 6378137.0
#define DGO_WGS84_F (1.0 / 298.257223563)
#define DGO_PI 3.14159265358979323846

typedef struct {
    double lat0_deg, lon0_deg; /* grid centre */
    double dlat_m, dlon_m;     /* node spacing in metres at the centre latitude */
    int32_t nlat, nlon;        /* row-major [lat][lon] */
} dgo_grid;

static double wgs84_e2(void) { return DGO_WGS84_F * (2.0 - DGO_WGS84_F); }

/* Sec. III: candidate points given in latitude/longitude on the ellipsoid,
 * converted to ECEF by the standard geodetic transformation. */
void dgo_geodetic_to_ecef(double lat_rad, double lon_rad, double h, double out[3])
{
    double e2 = wgs84_e2();
    double s = sin(lat_rad);
    double n = DGO_WGS84_A / sqrt(1.0 - e2 * s * s); /* prime-vertical radius */
    out[0] = (n + h) * cos(lat_rad) * cos(lon_rad);
    out[1] = (n + h) * cos(lat_rad) * sin(lon_rad);
    out[2] = (n * (1.0 - e2) + h) * s;
}

/* Angular node spacing of the grid: metres at the centre latitude divided by
 * the meridian radius (latitude) or the parallel's radius (longitude). */
void dgo_grid_step_rad(const dgo_grid *g, double *dlat_rad, double *dlon_rad)
{
    double e2 = wgs84_e2();
    double phi0 = g->lat0_deg * (DGO_PI / 180.0);
    double s = sin(phi0);
    double w = sqrt(1.0 - e2 * s * s);
    double m = DGO_WGS84_A * (1.0 - e2) / (w * w * w); /* meridian radius */
    double n = DGO_WGS84_A / w;                         /* prime vertical */
    *dlat_rad = g->dlat_m / m;
    *dlon_rad = g->dlon_m / (n * cos(phi0));
}

void dgo_grid_node(const dgo_grid *g, int64_t i, int64_t j, double *lat_rad, double *lon_rad)
{
    double dlat, dlon;
    dgo_grid_step_rad(g, &dlat, &dlon);
    *lat_rad = g->lat0_deg * (DGO_PI / 180.0) + ((double)i - 0.5 * (double)(g->nlat - 1)) * dlat;
    *lon_rad = g->lon0_deg * (DGO_PI / 180.0) + ((double)j - 0.5 * (double)(g->nlon - 1)) * dlon;
}

/* Algorithm 1, first step: every candidate to ECEF. xyz is [G][3]. */
void dgo_grid_ecef(const dgo_grid *g, double *xyz)
{
    for (int64_t i = 0; i < g->nlat; ++i)
        for (int64_t j = 0; j < g->nlon; ++j) {
            double lat, lon;
            dgo_grid_node(g, i, j, &lat, &lon);
            dgo_geodetic_to_ecef(lat, lon, 0.0, xyz + 3 * (i * (int64_t)g->nlon + j));
        }
}

/* Eq. 3-8 for one candidate pc and one snapshot's receiver states
 * eph = [p1 v1 p2 v2] (ECEF, m and m/s), receivers i=1, j=2.
 * out = [dtau (s), dfreq (Hz), D = dtau*fs (samples), nu = dfreq/fs]. */
void dgo_geometry(const double pc[3], const double eph[12], double fs, double fc, double out[4])
{
    const double *p1 = eph, *v1 = eph + 3, *p2 = eph + 6, *v2 = eph + 9;
    double lambda = DGO_C_LIGHT / fc;
    /* Eq. 3: r_i = p_i - p_e */
    double r1x = p1[0] - pc[0], r1y = p1[1] - pc[1], r1z = p1[2] - pc[2];
    double r2x = p2[0] - pc[0], r2y = p2[1] - pc[1], r2z = p2[2] - pc[2];
    /* Eq. 4: rho_i = sqrt(r_i^T r_i) = c tau_i */
    double rho1 = sqrt((r1x * r1x + r1y * r1y) + r1z * r1z);
    double rho2 = sqrt((r2x * r2x + r2y * r2y) + r2z * r2z);
    /* Eq. 5-6: f_i = -(1/lambda) rhat_i^T v_i = -(r_i^T v_i) / (rho_i lambda) */
    double f1 = -((r1x * v1[0] + r1y * v1[1]) + r1z * v1[2]) / (rho1 * lambda);
    double f2 = -((r2x * v2[0] + r2y * v2[1]) + r2z * v2[2]) / (rho2 * lambda);
    /* Eq. 7-8 with i = 1, j = 2 */
    double dtau = (rho2 - rho1) / DGO_C_LIGHT;
    double dfreq = f2 - f1;
    out[0] = dtau;
    out[1] = dfreq;
    out[2] = dtau * fs; /* Eq. 9 before rounding, in samples */
    out[3] = dfreq / fs;
}

/* Cubic Lagrange weights for taps at offsets -1, 0, 1, 2 evaluated at mu. */
void dgo_lagrange4(double mu, double w[4])
{
    w[0] = -mu * (mu - 1.0) * (mu - 2.0) / 6.0;
    w[1] = (mu + 1.0) * (mu - 1.0) * (mu - 2.0) / 2.0;
    w[2] = -(mu + 1.0) * mu * (mu - 2.0) / 2.0;
    w[3] = (mu + 1.0) * mu * (mu - 1.0) / 6.0;
}

/* Eq. 11 before the magnitude: C = sum_k y1[k] conj(y2~[k]) exp(j 2 pi nu k),
 * y2~[k] = y2[k + L] (delay_mode 0, L = round(D)) or the 4-tap Lagrange
 * interpolation of y2 at k + D (delay_mode 1, L = floor(D)).
 * y1, y2 are [n][2] (re, im). out = [re, im]. */
void dgo_correlate(const double *y1, const double *y2, int64_t n, double D, double nu,
                   int delay_mode, double out[2])
{
    double acc_re = 0.0, acc_im = 0.0;
    int64_t L;
    double w[4] = {0.0, 1.0, 0.0, 0.0};
    if (delay_mode == 0) {
        L = (int64_t)llround(D);
    } else {
        L = (int64_t)floor(D);
        dgo_lagrange4(D - (double)L, w);
    }
    for (int64_t k = 0; k < n; ++k) {
        double b_re = 0.0, b_im = 0.0; /* y2~[k] */
        for (int m = -1; m <= 2; ++m) {
            if (w[m + 1] == 0.0 && delay_mode == 0) continue;
            int64_t q = k + L + m;
            if (q < 0 || q >= n) continue;
            b_re += w[m + 1] * y2[2 * q];
            b_im += w[m + 1] * y2[2 * q + 1];
        }
        double a_re = y1[2 * k], a_im = y1[2 * k + 1];
        /* y1 * conj(y2~) */
        double p_re = a_re * b_re + a_im * b_im;
        double p_im = a_im * b_re - a_re * b_im;
        /* exp(j 2 pi nu k), phase reduced modulo one cycle */
        double ph = nu * (double)k;
        double ang = 2.0 * DGO_PI * (ph - floor(ph));
        double e_re = cos(ang), e_im = sin(ang);
        acc_re += p_re * e_re - p_im * e_im;
        acc_im += p_re * e_im + p_im * e_re;
    }
    out[0] = acc_re;
    out[1] = acc_im;
}

/* Algorithm 1 for a list of candidate indices: per candidate, for each
 * snapshot in order, geometry -> correlation -> |C|^2 (acc_mode 0) or |C|
 * (acc_mode 1), summed over snapshots in order k = 0..K-1.
 * eph is [K][12], y1/y2 are [K][N][2]. cost is [npts]. Optional outputs
 * (may be NULL): corr [npts][K][2] complex C_k, geom [npts][K][4]. */
int dgo_cost_points(const dgo_grid *g, const double *eph, int32_t K, double fs, double fc,
                    const double *y1, const double *y2, int64_t N, int delay_mode, int acc_mode,
                    const int64_t *idx, int64_t npts, double *cost, double *corr, double *geom,
                    int nthreads)
{
    if (!g || !eph || !y1 || !y2 || !idx || !cost || K < 1 || N < 1 || npts < 0) return 1;
    if (delay_mode != 0 && delay_mode != 1) return 1;
    if (acc_mode != 0 && acc_mode != 1) return 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int64_t G = (int64_t)g->nlat * g->nlon;
    for (int64_t p = 0; p < npts; ++p)
        if (idx[p] < 0 || idx[p] >= G) return 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t p = 0; p < npts; ++p) {
        int64_t i = idx[p] / g->nlon, j = idx[p] % g->nlon;
        double lat, lon, pc[3];
        dgo_grid_node(g, i, j, &lat, &lon);
        dgo_geodetic_to_ecef(lat, lon, 0.0, pc);
        double s = 0.0;
        for (int32_t k = 0; k < K; ++k) {
            double geo[4], c[2];
            dgo_geometry(pc, eph + 12 * (int64_t)k, fs, fc, geo);
            dgo_correlate(y1 + 2 * N * (int64_t)k, y2 + 2 * N * (int64_t)k, N, geo[2], geo[3],
                          delay_mode, c);
            double pw = c[0] * c[0] + c[1] * c[1];
            s += (acc_mode == 0) ? pw : sqrt(pw);
            if (corr) {
                corr[2 * (p * K + k)] = c[0];
                corr[2 * (p * K + k) + 1] = c[1];
            }
            if (geom) memcpy(geom + 4 * (p * K + k), geo, sizeof geo);
        }
        cost[p] = s;
    }
    return 0;
}

/* Eq. 3-10 at every node of a grid for K snapshots: D[k][p] = dtau * fs
 * (samples) and nu[k][p] = dfreq / fs (cycles per sample), p = i * nlon + j.
 * Returns 0, or -1 if the scratch allocation fails. */
int dgo_node_geometry(const dgo_grid *g, const double *eph, int32_t K, double fs, double fc, double *D,
                      double *nu)
{
    const int64_t G = (int64_t)g->nlat * g->nlon;
    double *xyz = (double *)malloc(sizeof(double) * 3 * (size_t)(G > 0 ? G : 1));
    if (!xyz) return -1;
    dgo_grid_ecef(g, xyz);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < G; ++p)
        for (int32_t k = 0; k < K; ++k) {
            double geo[4];
            dgo_geometry(xyz + 3 * p, eph + 12 * (int64_t)k, fs, fc, geo);
            D[k * G + p] = geo[2];
            nu[k * G + p] = geo[3];
        }
    free(xyz);
    return 0;
}

/* Maximum with ties broken by the lowest index; NaN never wins. -1 if none. */
int64_t dgo_argmax(const double *cost, int64_t n)
{
    int64_t best = -1;
    for (int64_t p = 0; p < n; ++p)
        if (cost[p] == cost[p] && (best < 0 || cost[p] > cost[best])) best = p;
    return best;
}

/* Algorithm 1, last step: threshold detection of emitters on an accumulated
 * surface [nlat][nlon]. A node is reported when its value is >= threshold and
 * it is the maximum of the (2r+1) x (2r+1) window of nodes around it (within
 * the grid); among equal values the lowest linear index wins, so a plateau
 * yields one peak. Peaks are ordered by value, descending, ties by index;
 * at most max_peaks are written to idx. Returns the number written. */
int64_t dgo_detect(const double *v, int32_t nlat, int32_t nlon, double threshold, int32_t r,
                   int64_t max_peaks, int64_t *idx)
{
    int64_t n = 0, cap = max_peaks;
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)((int64_t)nlat * nlon + 1));
    if (!tmp) return -1;
    for (int64_t i = 0; i < nlat; ++i)
        for (int64_t j = 0; j < nlon; ++j) {
            int64_t p = i * nlon + j;
            double x = v[p];
            if (!(x >= threshold)) continue;
            int peak = 1;
            for (int64_t di = -r; di <= r && peak; ++di)
                for (int64_t dj = -r; dj <= r; ++dj) {
                    int64_t ii = i + di, jj = j + dj;
                    if ((di == 0 && dj == 0) || ii < 0 || jj < 0 || ii >= nlat || jj >= nlon) continue;
                    int64_t q = ii * nlon + jj;
                    if (v[q] > x || (v[q] == x && q < p)) {
                        peak = 0;
                        break;
                    }
                }
            if (peak) tmp[n++] = p;
        }
    /* insertion sort by (value desc, index asc): peaks are few */
    for (int64_t a = 1; a < n; ++a) {
        int64_t key = tmp[a], b = a - 1;
        while (b >= 0 && (v[tmp[b]] < v[key] || (v[tmp[b]] == v[key] && tmp[b] > key))) {
            tmp[b + 1] = tmp[b];
            --b;
        }
        tmp[b + 1] = key;
    }
    if (n > cap) n = cap;
    memcpy(idx, tmp, sizeof(int64_t) * (size_t)n);
    free(tmp);
    return n;
}
