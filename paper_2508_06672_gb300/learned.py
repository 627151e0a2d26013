"""Learned proposal search over a large footprint.

The full-grid search (Algorithm 1 on every node of the footprint, then a
dense re-evaluation around the argmax) is replaced by:

1. coarse per-snapshot delay-Doppler maps back-projected onto the footprint's
   cells (dg_coarse_maps), K channels;
2. a small convolutional network (ProposalNet, the library's own kernels)
   turning them into one map of logits, the belief that the emitter sits in
   each cell;
3. the top ``regions`` cells of that map, at least ``2 radius + 1`` cells
   apart (dg_detect on the cell-centre grid);
4. around each, the cost surface of Algorithm 1 on the full search's nodes
   within a square of side ``region_m``, its argmax and the same dense
   re-evaluation as the full search (dg_set_grid, dg_search_regions on one
   context that keeps the captures);
5. the region whose argmax holds the largest cost gives the fix;
6. the full-grid search on the same context is the fallback: it runs when
   no region is proposed, when the winning region's argmax lies within
   ``edge`` nodes of the region's border (the surface still rises towards
   the border, so the maximum may lie outside every region), or when the
   search looks unsure: the best proposal's logit is below ``min_logit`` or
   the best region's maximum exceeds the runner-up's by less than
   ``min_region_gap`` of it.

The method without the network ranks the cells by the sum of the K coarse
maps instead (the non-coherent sum of Algorithm 1 applied to the coarse
maps); ``SumNet`` is that sum as a fixed 3 x 3 convolution.
"""
from __future__ import annotations

import math

import numpy as np

from . import dg
from .proposal import ProposalNet


def footprint_grids(grid, cells):
    """(node grid, cell-centre grid) of ``cells`` x ``cells`` coarse cells
    covering the footprint of ``grid`` (same centre, same side)."""
    side_lat = (int(grid["nlat"]) - 1) * float(grid["dlat_m"])
    side_lon = (int(grid["nlon"]) - 1) * float(grid["dlon_m"])
    base = dict(lat0_deg=float(grid["lat0_deg"]), lon0_deg=float(grid["lon0_deg"]),
                dlat_m=side_lat / cells, dlon_m=side_lon / cells)
    return dict(base, nlat=cells + 1, nlon=cells + 1), dict(base, nlat=cells, nlon=cells)


def degrees_per_metre(lat_deg):
    """WGS-84 degrees of latitude and longitude per metre at lat_deg (the
    meridian and prime-vertical radii), as the grids use them."""
    a, f = 6378137.0, 1.0 / 298.257223563
    e2 = f * (2.0 - f)
    s = math.sin(math.radians(lat_deg))
    w = math.sqrt(1.0 - e2 * s * s)
    return math.degrees(w ** 3 / (a * (1.0 - e2))), math.degrees(w / (a * math.cos(math.radians(lat_deg))))


def node_of(grid, lat_deg, lon_deg):
    """Fractional (row, column) of a point in a grid's node lattice."""
    dlat, dlon = degrees_per_metre(float(grid["lat0_deg"]))
    i = (lat_deg - float(grid["lat0_deg"])) / (dlat * float(grid["dlat_m"])) + 0.5 * (int(grid["nlat"]) - 1)
    j = (lon_deg - float(grid["lon0_deg"])) / (dlon * float(grid["dlon_m"])) + 0.5 * (int(grid["nlon"]) - 1)
    return i, j


def distance_m(lat1, lon1, lat2, lon2):
    """Great-circle distance on the sphere of radius 6371 km."""
    p1, p2 = math.radians(lat1), math.radians(lat2)
    dp, dl = p2 - p1, math.radians(lon2 - lon1)
    h = math.sin(dp / 2) ** 2 + math.cos(p1) * math.cos(p2) * math.sin(dl / 2) ** 2
    return 2 * 6371e3 * math.asin(min(1.0, math.sqrt(h)))


class SumNet:
    """The method without the network: the sum of the K coarse maps, as a
    fixed 3 x 3 convolution (centre tap 1 for every channel)."""

    def __init__(self, K, device="cuda"):
        import torch
        w = np.zeros((1, K, 3, 3))
        w[0, :, 1, 1] = 1.0
        self.net = ProposalNet([K, 1], device=device)
        self.net.load_numpy([(w, np.zeros(1))])
        self.torch = torch

    def forward(self, x, keep=False):
        return self.net.forward(x)


class LearnedSearch:
    """The learned search of one footprint (``grid``: the full search's grid,
    whose node spacing the regions reuse)."""

    def __init__(self, grid, ephem, fs_hz, fc_hz, net, *, cells=512, regions=8, region_m=50e3,
                 refine_spacing_m=25.0, refine_window_m=500.0, bins=0, chunk=0, algo="cdft",
                 contract="bf16x3", stream=None, edge=2, min_logit=3.6, min_region_gap=0.2):
        import torch
        self.torch = torch
        self.grid = dict(grid)
        self.net = net
        self.cells = int(cells)
        self.regions = int(regions)
        self.node_grid, self.centre_grid = footprint_grids(grid, self.cells)
        cell_m = float(self.node_grid["dlat_m"])
        self.radius = max(1, int(math.ceil(0.5 * region_m / cell_m)))
        self.half = int(round(0.5 * region_m / float(grid["dlat_m"])))
        self.refine = (float(refine_spacing_m), float(refine_window_m))
        self.bins, self.chunk = int(bins), int(chunk)
        eph = np.ascontiguousarray(ephem, dtype=np.float64).reshape(-1, 12)
        self.K = eph.shape[0]
        self.geo = dg.Geolocator(self.node_grid, eph, fs_hz, fc_hz, algo=algo, contract=contract,
                                 stream=stream)
        self.hm = dg.Geolocator(self.centre_grid, eph, fs_hz, fc_hz, stream=self.geo.stream)
        self.maps = torch.empty((self.K, self.cells, self.cells), dtype=torch.float32, device=self.geo.device)
        self.cost = None
        self.full_cost = None
        self.edge = int(edge)
        # Unsure-search thresholds of the fallback. The defaults are the 2nd
        # percentiles, over the shipped network's successful searches on the
        # training script's 200 held-out scenes (seeds 5, 100005...), of the
        # best proposal's logit (3.6) and of the relative margin of the best
        # region's maximum over the runner-up's (0.2): about 4 % of searches
        # fall back. They belong to those weights (the logit scale is the
        # network's); None switches a criterion off.
        self.min_logit = min_logit
        self.min_region_gap = min_region_gap
        self.searches = 0     # search() calls, and how many of them fell back to the full grid
        self.fallbacks = 0
        self.fell_back = False

    def load_captures(self, fmt, y1, y2):
        self.geo.load_captures(fmt, y1, y2)

    def coarse(self):
        """The K coarse maps of the footprint (device, K x cells x cells)."""
        self.geo.set_grid(self.node_grid)
        return self.geo.coarse_maps(bins=self.bins, chunk=self.chunk, out=self.maps)

    def heatmap(self, net=None):
        maps = self.coarse()
        with self.torch.cuda.stream(self.geo.stream):
            return (net or self.net).forward(maps.view(1, self.K, self.cells, self.cells))

    def proposals(self, net=None):
        """The top cells as dg_peak dicts (lat_deg, lon_deg, value, i, j)."""
        logits = self.heatmap(net).view(self.cells, self.cells)
        # dg_detect returns the largest local maxima however many there are
        return self.hm.detect(logits, -3.0e38, relative=False, radius=self.radius, max_peaks=self.regions)

    def region_grid(self, lat_deg, lon_deg):
        """The region around a point: the nodes of the full search's grid
        within ``half`` rows and columns of the node nearest to the point.
        A grid's node spacing is set in metres and turned into degrees at its
        own centre latitude, so the region takes the spacing in metres that
        gives the full grid's degree steps at the region's centre: its nodes
        are then nodes of the full grid."""
        i, j = node_of(self.grid, lat_deg, lon_deg)
        i = min(max(int(round(i)), 0), int(self.grid["nlat"]) - 1)
        j = min(max(int(round(j)), 0), int(self.grid["nlon"]) - 1)
        dlat0, dlon0 = degrees_per_metre(float(self.grid["lat0_deg"]))
        step_lat = dlat0 * float(self.grid["dlat_m"])  # degrees per row and per column of the full grid
        step_lon = dlon0 * float(self.grid["dlon_m"])
        lat = float(self.grid["lat0_deg"]) + (i - 0.5 * (int(self.grid["nlat"]) - 1)) * step_lat
        lon = float(self.grid["lon0_deg"]) + (j - 0.5 * (int(self.grid["nlon"]) - 1)) * step_lon
        dlat, dlon = degrees_per_metre(lat)
        n = 2 * self.half + 1
        return dict(lat0_deg=lat, lon0_deg=lon, dlat_m=step_lat / dlat, dlon_m=step_lon / dlon, nlat=n, nlon=n)

    def doubtful(self, fix):
        """True when a region's fix cannot be trusted: its argmax lies within
        ``edge`` nodes of the region's border."""
        n = 2 * self.half + 1
        return min(fix["i"], fix["j"], n - 1 - fix["i"], n - 1 - fix["j"]) < self.edge

    def unsure(self, peaks, costs):
        """True when the proposals do not single out a region: the best
        proposal's logit is under ``min_logit``, or the best region's
        maximum cost exceeds the runner-up's by less than ``min_region_gap``
        of it. ``costs``: the regions' cost surfaces (device)."""
        if self.min_logit is not None and max(p["value"] for p in peaks) < self.min_logit:
            return True
        if self.min_region_gap is not None and len(peaks) > 1:
            with self.torch.cuda.stream(self.geo.stream):
                top = self.torch.topk(costs.flatten(1).amax(1), 2).values.tolist()
            return top[0] - top[1] < self.min_region_gap * top[0]
        return False

    def full_search(self):
        """The full-grid search (Algorithm 1 on every node, then the same
        dense re-evaluation) on the same context and captures."""
        self.geo.set_grid(self.grid)
        if self.full_cost is None:
            self.full_cost = self.torch.empty((int(self.grid["nlat"]), int(self.grid["nlon"])),
                                              dtype=self.torch.float32, device=self.geo.device)
        self.geo.cost_surface(out=self.full_cost)
        return self.geo.argmax_refine(self.full_cost, *self.refine)

    def search(self, net=None, fallback=True):
        """(fix, index of the region it came from, proposals). With fallback,
        a search that proposes no region or whose fix is doubtful runs the
        full-grid search instead: its fix is returned with index -1 and
        ``fell_back`` is set. Without it, no proposal gives (None, -1, [])."""
        self.searches += 1
        self.fell_back = False
        peaks = self.proposals(net)
        if peaks:
            n = 2 * self.half + 1
            if self.cost is None:
                self.cost = self.torch.empty((self.regions, n, n), dtype=self.torch.float32, device=self.geo.device)
            regions = [self.region_grid(p["lat_deg"], p["lon_deg"]) for p in peaks]
            fix, best, costs = self.geo.search_regions(regions, *self.refine, costs=self.cost)
            if not fallback or not (self.doubtful(fix) or self.unsure(peaks, costs[:len(regions)])):
                return fix, best, peaks
        elif not fallback:
            return None, -1, peaks
        self.fallbacks += 1
        self.fell_back = True
        return self.full_search(), -1, peaks

    def close(self):
        self.geo.close()
        self.hm.close()


def cell_of(node_grid, lat_deg, lon_deg):
    """(row, column) of the coarse cell holding a point."""
    i, j = node_of(node_grid, lat_deg, lon_deg)
    return int(math.floor(i)), int(math.floor(j))


def target_map(cells, ci, cj, sigma=1.0):
    """Training target: a Gaussian bump of peak 1 on cell (ci, cj)."""
    ii, jj = np.mgrid[0:cells, 0:cells]
    t = np.exp(-0.5 * ((ii - ci) ** 2 + (jj - cj) ** 2) / sigma ** 2)
    t[t < 1e-3] = 0.0
    return t
