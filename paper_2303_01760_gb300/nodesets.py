"""Seeded synthetic node sets shaped like the paper's natural-convection domains.

Input data only.  This module builds node positions and per-node flags; it holds
none of the method's arithmetic (no stencil selection, no weights, no operator,
no time step).  Both the CUDA path and the CPU oracle consume its output.

Construction follows the hybrid fill of Section 2: the whole domain is first
covered by a regular lattice of spacing h, the lattice nodes where scattered
nodes are wanted (a band of width ``band`` around the irregular boundaries) are
removed, and the void is refilled with Poisson-disk scattered nodes of the same
spacing.  The paper's own positioning algorithm (a cited advancing-front fill)
and its duck-shaped obstacles are not available; circular / spherical holes and
a Bridson-style dart-throwing fill, both seeded, stand in for them.

The h-refined sets of Sections 4.2 and 4.3 (``holes_refined``) refill the
layer with a variable-density dart throwing instead: the spacing falls
linearly from the lattice spacing to a fraction of it at the obstacles, and
each node's spacing is kept in ``NodeSet.spacing``.

Node order: all nodes are sorted by the Morton code of their position at
resolution h (ties keep lattice-first construction order), which keeps stencil
neighbours close in memory.  Node ids are positions in that order.

Boundary conditions follow Section 4: de Vahl Davis walls (cold left, hot right,
insulated top/bottom) for the square, insulated box walls and alternating
cold/hot Dirichlet obstacles (T_C = 0 for even hole index, T_H = 1 for odd) for
the irregular domains.  Corner nodes (2D) and edge/corner nodes (3D) of the box
are dropped, which reproduces the paper's regular dVD count N = 253**2 - 4.
"""
from __future__ import annotations

import hashlib
import math
import os
from dataclasses import dataclass, field

import numpy as np

BC_INTERIOR = 0
BC_T_DIRICHLET = 1
BC_T_NEUMANN = 2

SEED_BASE = 20230301


@dataclass
class NodeSet:
    """A node set: SoA coordinates plus per-node flags.

    coords      float64 [dim, N]   node positions
    is_regular  uint8   [N]        1 = regular lattice node (candidate for MON)
    is_boundary uint8   [N]        1 = node lies on the domain boundary
    normals     float64 [dim, N]   outward unit normal of boundary nodes, 0 inside
    bc          uint8   [N]        BC_INTERIOR / BC_T_DIRICHLET / BC_T_NEUMANN
    T_bc        float64 [N]        Dirichlet temperature (0 where not Dirichlet)
    T_ref       float               reference temperature of the Boussinesq term
    spacing     float64 [N] or None local internodal distance h(x_i) of an
                                    h-refined set (None: h everywhere)
    """

    name: str
    dim: int
    h: float
    coords: np.ndarray
    is_regular: np.ndarray
    is_boundary: np.ndarray
    normals: np.ndarray
    bc: np.ndarray
    T_bc: np.ndarray
    T_ref: float
    holes: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    band: float = 0.0
    spacing: np.ndarray | None = None

    @property
    def N(self) -> int:
        return int(self.coords.shape[1])

    @property
    def n_scattered(self) -> int:
        return int(self.N - int(self.is_regular.sum()))

    def all_scattered(self) -> "NodeSet":
        """The same node set with every node flagged scattered (all RBF-FD)."""
        return NodeSet(self.name + "-allrbf", self.dim, self.h, self.coords,
                       np.zeros_like(self.is_regular), self.is_boundary,
                       self.normals, self.bc, self.T_bc, self.T_ref,
                       self.holes, self.band, self.spacing)


# --------------------------------------------------------------------------
# Poisson-disk fill (vectorised Bridson dart throwing with fixed pre-seeded
# samples).  A uniform grid with cell size h/sqrt(d) holds at most a few
# points per cell, so "is any point closer than h" is a fixed-size lookup.
# --------------------------------------------------------------------------
_SLOTS = 4


class _Grid:
    """``h`` is the smallest spacing (it sets the cell size); ``reach`` the
    largest distance a proximity query asks about (default h)."""

    def __init__(self, dim, h, lo, hi, reach=None):
        reach = h if reach is None else reach
        self.dim = dim
        self.h = h
        self.cell = h / math.sqrt(dim)
        self.lo = np.asarray(lo, dtype=np.float64)
        self.shape = np.ceil((np.asarray(hi) - self.lo) / self.cell).astype(np.int64) + 1
        self.ncell = int(np.prod(self.shape))
        self.slots = np.full((self.ncell, _SLOTS), -1, dtype=np.int64)
        self.fill = np.zeros(self.ncell, dtype=np.int64)
        r = int(math.ceil(reach / self.cell))
        rng = np.arange(-r, r + 1)
        offs = np.stack(np.meshgrid(*([rng] * dim), indexing="ij"), -1).reshape(-1, dim)
        # skip neighbour cells whose closest point is already >= reach away
        gap = np.maximum(np.abs(offs) - 1, 0) * self.cell
        self.offs = offs[np.sqrt((gap ** 2).sum(1)) < reach]
        self.pts = np.zeros((0, dim))
        self.rad = np.zeros(0)  # per-point exclusion radius (variable-density fills)

    def cell_of(self, p):
        c = np.floor((p - self.lo) / self.cell).astype(np.int64)
        return np.clip(c, 0, self.shape - 1)

    def lin(self, c):
        idx = c[..., 0]
        for k in range(1, self.dim):
            idx = idx * self.shape[k] + c[..., k]
        return idx

    def insert(self, p, rad=None):
        base = len(self.pts)
        self.pts = np.concatenate([self.pts, p], 0)
        self.rad = np.concatenate([self.rad, np.zeros(len(p)) if rad is None else rad])
        cid = self.lin(self.cell_of(p))
        order = np.argsort(cid, kind="stable")
        cs = cid[order]
        start = np.r_[0, np.flatnonzero(np.diff(cs)) + 1]
        rank = np.arange(len(cs)) - np.repeat(start, np.diff(np.r_[start, len(cs)]))
        slot = self.fill[cs] + rank
        if len(slot) and slot.max() >= _SLOTS:
            raise RuntimeError("Poisson-disk grid overflow: fixed nodes closer than the fill spacing")
        self.slots[cs, slot] = base + order
        np.add.at(self.fill, cs, 1)

    def too_close(self, p, chunk=1 << 16, radius=None):
        """Whether a stored point lies closer than h to each p[i]; with
        ``radius`` (per query point, up to ``reach``) closer than the larger of
        radius[i] and the stored point's own radius."""
        out = np.zeros(len(p), dtype=bool)
        if radius is not None:
            chunk = max(256, (1 << 22) // (len(self.offs) * _SLOTS))
        for s in range(0, len(p), chunk):
            q = p[s:s + chunk]
            c = self.cell_of(q)
            nb = c[:, None, :] + self.offs[None, :, :]
            ok = np.all((nb >= 0) & (nb < self.shape), axis=-1)
            nb = np.clip(nb, 0, self.shape - 1)
            ids = self.slots[self.lin(nb)]             # [m, offs, slots]
            ids = np.where(ok[..., None], ids, -1).reshape(len(q), -1)
            valid = ids >= 0
            pp = self.pts[np.where(valid, ids, 0)]     # [m, k, dim]
            d2 = ((pp - q[:, None, :]) ** 2).sum(-1)
            if radius is None:
                lim = self.h * self.h
            else:
                lim = np.maximum(radius[s:s + chunk][:, None], self.rad[np.where(valid, ids, 0)]) ** 2
            out[s:s + chunk] = np.any(valid & (d2 < lim), axis=1)
        return out


def _poisson_fill(fixed, seeds, accept, h, lo, hi, rng, k):
    """Fill the region where ``accept(p)`` holds with points >= h apart from each
    other and from ``fixed``; dart throwing starts from ``seeds``."""
    from scipy.spatial import cKDTree

    dim = fixed.shape[1]
    g = _Grid(dim, h, lo, hi)
    g.insert(fixed)
    n_fixed = len(fixed)
    active = np.asarray(seeds, dtype=np.float64)
    while len(active):
        m = len(active)
        if dim == 2:
            th = rng.uniform(0.0, 2.0 * math.pi, (m, k))
            dirs = np.stack([np.cos(th), np.sin(th)], -1)
        else:
            dirs = rng.normal(size=(m, k, dim))
            dirs /= np.linalg.norm(dirs, axis=-1, keepdims=True)
        rad = h * rng.uniform(1.0, 2.0, (m, k, 1))
        cand = (active[:, None, :] + rad * dirs).reshape(-1, dim)
        inside = np.all((cand > lo) & (cand < hi), axis=1)
        ok = inside.copy()
        ok[inside] = accept(cand[inside])
        ok[ok] = ~g.too_close(cand[ok])
        alive = ok.reshape(m, k).any(1)
        c_idx = np.flatnonzero(ok)
        cands = cand[c_idx]
        if len(cands):
            pri = rng.random(len(cands))
            pairs = cKDTree(cands).query_pairs(h * (1.0 - 1e-12), output_type="ndarray")
            lose = np.zeros(len(cands), dtype=bool)
            if len(pairs):
                i, j = pairs[:, 0], pairs[:, 1]
                first_loses = pri[i] > pri[j]
                lose[i[first_loses]] = True
                lose[j[~first_loses]] = True
            new = cands[~lose]
            g.insert(new)
        else:
            new = np.zeros((0, dim))
        active = np.concatenate([active[alive], new], 0)
    return g.pts[n_fixed:]


def _poisson_fill_var(fixed, fixed_rad, seeds, accept, hfun, h_min, h_max, lo, hi, rng, k):
    """Variable-density dart throwing (the h-refined fills of Sections 4.2 and
    4.3): darts from an active point a land at distances h(a)..2h(a).  Every
    point keeps its own exclusion disk (radius h(q) for a dart, ``fixed_rad``
    for the fixed nodes): a dart q is kept when no point p lies closer than
    max(h(q), r_p), so darts cannot squeeze between fixed nodes spaced wider
    than the local h, and keeps h(q)/2 from the box faces; of two kept darts
    closer than the larger of their spacings, the one of lower random
    priority goes."""
    from scipy.spatial import cKDTree

    dim = fixed.shape[1]
    g = _Grid(dim, h_min, lo, hi, reach=h_max)
    g.insert(fixed, fixed_rad)
    n_fixed = len(fixed)
    active = np.asarray(seeds, dtype=np.float64)
    while len(active):
        m = len(active)
        if dim == 2:
            th = rng.uniform(0.0, 2.0 * math.pi, (m, k))
            dirs = np.stack([np.cos(th), np.sin(th)], -1)
        else:
            dirs = rng.normal(size=(m, k, dim))
            dirs /= np.linalg.norm(dirs, axis=-1, keepdims=True)
        rad = hfun(active)[:, None, None] * rng.uniform(1.0, 2.0, (m, k, 1))
        cand = (active[:, None, :] + rad * dirs).reshape(-1, dim)
        # half a local spacing clear of the box faces: keeps darts out of the
        # empty channels along box edges (edge lattice nodes are dropped)
        inside = np.min(np.minimum(cand - lo, hi - cand), axis=1) >= 0.5 * hfun(cand)
        ok = inside.copy()
        ok[inside] = accept(cand[inside])
        ok[ok] = ~g.too_close(cand[ok], radius=hfun(cand[ok]))
        alive = ok.reshape(m, k).any(1)
        cands = cand[np.flatnonzero(ok)]
        if len(cands):
            pri = rng.random(len(cands))
            hc = hfun(cands)
            pairs = cKDTree(cands).query_pairs(h_max, output_type="ndarray")
            lose = np.zeros(len(cands), dtype=bool)
            if len(pairs):
                i, j = pairs[:, 0], pairs[:, 1]
                dd = np.sqrt(((cands[i] - cands[j]) ** 2).sum(1))
                clash = dd < np.maximum(hc[i], hc[j]) * (1.0 - 1e-12)
                i, j = i[clash], j[clash]
                first_loses = pri[i] > pri[j]
                lose[i[first_loses]] = True
                lose[j[~first_loses]] = True
            new = cands[~lose]
            g.insert(new, hc[~lose])
        else:
            new = np.zeros((0, dim))
        active = np.concatenate([active[alive], new], 0)
    return g.pts[n_fixed:]


# --------------------------------------------------------------------------
# Geometry helpers
# --------------------------------------------------------------------------
def _lattice(dim, n):
    ax = np.arange(n + 1)
    ijk = np.stack(np.meshgrid(*([ax] * dim), indexing="ij"), 0).reshape(dim, -1)
    # x fastest: meshgrid 'ij' gives first axis slowest, so reverse the axis order
    ijk = ijk[::-1].copy()
    return ijk


def _place_holes(dim, n_holes, r_range, gap, margin, rng, max_tries=200000):
    holes = []
    tries = 0
    while len(holes) < n_holes:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place holes")
        r = rng.uniform(*r_range)
        c = rng.uniform(r + margin, 1.0 - r - margin, dim)
        if all(np.linalg.norm(c - hc[:dim]) >= r + hc[dim] + gap for hc in holes):
            holes.append(np.r_[c, r])
    return np.array(holes).reshape(n_holes, dim + 1)


def _hole_surface(dim, c, r, h, rng):
    if dim == 2:
        nb = max(8, int(math.floor(2.0 * math.pi * r / h)))
        th = rng.uniform(0, 2 * math.pi) + 2.0 * math.pi * np.arange(nb) / nb
        u = np.stack([np.cos(th), np.sin(th)], 0)
    else:
        # Fibonacci sphere with about one node per 1.25 h^2 of surface
        nb = max(12, int(math.floor(4.0 * math.pi * r * r / (1.25 * h * h))))
        i = np.arange(nb) + 0.5
        phi = np.arccos(1.0 - 2.0 * i / nb)
        th = math.pi * (1.0 + math.sqrt(5.0)) * i + rng.uniform(0, 2 * math.pi)
        u = np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 0)
    x = c[:, None] + r * u
    return x, -u  # outward normal of the fluid domain points into the hole


def _morton_order(coords, h):
    dim = coords.shape[0]
    q = np.floor(coords / h + 0.5).astype(np.int64)
    q = np.clip(q, 0, (1 << 20) - 1)
    code = np.zeros(coords.shape[1], dtype=np.int64)
    bits = 20 if dim == 2 else 20
    for b in range(bits):
        for k in range(dim):
            code |= ((q[k] >> b) & 1) << (b * dim + k)
    return np.argsort(code, kind="stable")


def _min_hole_gap(x, holes, dim):
    """Distance from points x [m, dim] to the nearest hole surface."""
    if len(holes) == 0:
        return np.full(len(x), np.inf)
    c = holes[:, :dim]
    r = holes[:, dim]
    d = np.sqrt(((x[:, None, :] - c[None]) ** 2).sum(-1)) - r[None]
    return d.min(1)


def _build(name, dim, n, holes, band, wall_band, seed, bc_walls, hole_T, T_ref, k=None, region=None,
           hfun=None, h_min=None):
    """Common hybrid construction (Section 2): lattice, removal, Poisson refill.
    ``region(p)`` (optional) marks further points whose neighbourhood is
    discretised with scattered nodes.  ``hfun(p)`` (optional) is a spacing
    function for an h-refined fill, between ``h_min`` (on the hole surfaces)
    and the lattice spacing."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    ijk = _lattice(dim, n)
    x = ijk.T / n
    on_wall = (ijk == 0) | (ijk == n)
    n_wall = on_wall.sum(0)
    keep = n_wall <= 1
    gap = _min_hole_gap(x, holes, dim)
    wall_dist = np.minimum(x, 1.0 - x).min(1)
    eps = 1e-9 * h
    in_band_lat = (gap < band - eps) | (wall_dist < wall_band - eps)
    if region is not None:
        in_band_lat |= region(x)
    interior_lat = keep & (n_wall == 0) & ~in_band_lat & (gap > 0)
    wall_lat = keep & (n_wall == 1) & (gap > 0.5 * h)
    lat_pts = x[interior_lat | wall_lat]
    lat_is_wall = wall_lat[interior_lat | wall_lat]
    lat_ijk = ijk[:, interior_lat | wall_lat]

    hole_pts, hole_nrm, hole_id = [], [], []
    for hid, hc in enumerate(holes):
        p, nr = _hole_surface(dim, hc[:dim], hc[dim], h if hfun is None else h_min, rng)
        hole_pts.append(p.T)
        hole_nrm.append(nr.T)
        hole_id.append(np.full(p.shape[1], hid))
    hole_pts = np.concatenate(hole_pts, 0) if hole_pts else np.zeros((0, dim))
    hole_nrm = np.concatenate(hole_nrm, 0) if hole_nrm else np.zeros((0, dim))
    hole_id = np.concatenate(hole_id) if hole_id else np.zeros(0, dtype=np.int64)

    def accept(p):
        g = _min_hole_gap(p, holes, dim) if len(holes) else np.full(len(p), np.inf)
        wd = np.minimum(p, 1.0 - p).min(1)
        inside = (g < band - eps) | (wd < wall_band - eps)
        if region is not None:
            inside = inside | region(p)
        return (g > 0) & inside

    fixed = np.concatenate([lat_pts, hole_pts], 0)
    grow = 2.0 * h
    fixed_gap = _min_hole_gap(fixed, holes, dim)
    fixed_wd = np.minimum(fixed, 1.0 - fixed).min(1)
    near = (fixed_gap < band + grow) | (fixed_wd < wall_band + grow)
    if region is not None:
        # fixed points within 2h of the region seed its fill
        near |= region(fixed)
        for a in range(dim):
            for sgn in (-1.0, 1.0):
                q = fixed.copy()
                q[:, a] += sgn * grow
                near |= region(q)
    seeds = fixed[near]
    if k is None:
        k = 16 if dim == 2 else 10
    if hfun is None:
        scat = _poisson_fill(fixed, seeds, accept, h, np.zeros(dim), np.ones(dim), rng, k)
    else:
        # lattice and wall nodes keep the lattice spacing, hole nodes h_min
        fixed_rad = np.r_[np.full(len(lat_pts), h), np.full(len(hole_pts), h_min)]
        scat = _poisson_fill_var(fixed, fixed_rad, seeds, accept, hfun, h_min, h, np.zeros(dim), np.ones(dim), rng,
                                 k)

    N = len(fixed) + len(scat)
    coords = np.concatenate([fixed, scat], 0).T.copy()
    n_lat = len(lat_pts)
    n_hole = len(hole_pts)
    is_regular = np.zeros(N, dtype=np.uint8)
    is_regular[:n_lat] = (~lat_is_wall).astype(np.uint8)
    is_boundary = np.zeros(N, dtype=np.uint8)
    is_boundary[:n_lat] = lat_is_wall
    is_boundary[n_lat:n_lat + n_hole] = 1
    normals = np.zeros((dim, N))
    bc = np.zeros(N, dtype=np.uint8)
    T_bc = np.zeros(N)
    # box walls
    wi = np.flatnonzero(lat_is_wall)
    for node in wi:
        a = int(np.flatnonzero((lat_ijk[:, node] == 0) | (lat_ijk[:, node] == n))[0])
        side = 1 if lat_ijk[a, node] == n else 0
        normals[a, node] = 1.0 if side else -1.0
        kind, val = bc_walls(a, side)
        bc[node] = kind
        T_bc[node] = val
    # holes
    sl = slice(n_lat, n_lat + n_hole)
    normals[:, sl] = hole_nrm.T
    bc[sl] = BC_T_DIRICHLET
    T_bc[sl] = np.array([hole_T(int(i)) for i in hole_id]) if n_hole else 0.0

    order = _morton_order(coords, h)
    # each node's spacing: its exclusion radius in the fill
    spacing = None if hfun is None else np.r_[fixed_rad, hfun(scat)][order].copy()
    return NodeSet(name, dim, h, coords[:, order].copy(), is_regular[order].copy(),
                   is_boundary[order].copy(), normals[:, order].copy(), bc[order].copy(),
                   T_bc[order].copy(), T_ref, np.asarray(holes, dtype=np.float64), band, spacing)


# --------------------------------------------------------------------------
# The workloads
# --------------------------------------------------------------------------
def square_wall_band(n=40, wall_band=0.1, seed=SEED_BASE + 0):
    """Unit square, regular lattice h=1/n inside, Poisson-disk scattered nodes in
    a band of width ``wall_band`` along the walls; de Vahl Davis walls (Section
    4.1): T_C=-0.5 at x=0, T_H=+0.5 at x=1, insulated top and bottom."""

    def bc_walls(axis, side):
        if axis == 0:
            return BC_T_DIRICHLET, (0.5 if side else -0.5)
        return BC_T_NEUMANN, 0.0

    return _build(f"square-wallband-n{n}", 2, n, np.zeros((0, 3)), 0.0, wall_band, seed,
                  bc_walls, lambda i: 0.0, 0.0)


def square_quarters(n=100, layout="hybrid", seed=SEED_BASE + 5):
    """The de Vahl Davis square split into quarters, each discretised with
    either scattered or regular nodes (Section 4.1).  ``layout``: "hybrid"
    (bottom-left and top-right quarters scattered, the other two regular),
    "scattered" (all four) or "regular" (none).  Walls as in
    ``square_wall_band``: T_C = -0.5 at x = 0, T_H = +0.5 at x = 1, insulated
    top and bottom."""

    def bc_walls(axis, side):
        if axis == 0:
            return BC_T_DIRICHLET, (0.5 if side else -0.5)
        return BC_T_NEUMANN, 0.0

    if layout == "hybrid":
        def region(p):
            lo = (p[:, 0] < 0.5) & (p[:, 1] < 0.5)
            hi = (p[:, 0] >= 0.5) & (p[:, 1] >= 0.5)
            return lo | hi
        return _build(f"square-quarters-n{n}", 2, n, np.zeros((0, 3)), 0.0, 0.0, seed, bc_walls,
                      lambda i: 0.0, 0.0, region=region)
    if layout == "scattered":
        return _build(f"square-scattered-dvd-n{n}", 2, n, np.zeros((0, 3)), 0.0, 1.0, seed, bc_walls,
                      lambda i: 0.0, 0.0)
    if layout == "regular":
        return _build(f"square-regular-n{n}", 2, n, np.zeros((0, 3)), 0.0, 0.0, seed, bc_walls,
                      lambda i: 0.0, 0.0)
    raise ValueError(layout)


def square_holes(n=500, n_holes=8, r_range=(0.03, 0.08), band=0.05, seed=SEED_BASE + 1,
                 hole_gap=None):
    """Unit square minus ``n_holes`` seeded circular holes (Section 4.2 shape with
    circles standing in for the obstacles); scattered nodes within ``band`` of a
    hole, regular lattice h=1/n elsewhere.  Box insulated; holes alternate
    T_C=0 / T_H=1."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    gap = 2.0 * 0.05 if hole_gap is None else hole_gap
    holes = _place_holes(2, n_holes, r_range, gap, 2 * h, rng)

    def bc_walls(axis, side):
        return BC_T_NEUMANN, 0.0

    return _build(f"square-holes-n{n}-b{band:g}", 2, n, holes, band, 0.0, seed + 1000,
                  bc_walls, lambda i: float(i % 2), 0.5)


def cube_spheres(n=125, n_holes=20, r_range=(0.03, 0.08), band=0.05, seed=SEED_BASE + 2,
                 hole_gap=None):
    """Unit cube minus ``n_holes`` seeded spheres (Section 4.3 shape); scattered
    nodes within ``band`` of a sphere, regular lattice h=1/n elsewhere.  Box
    insulated; spheres alternate T_C=0 / T_H=1."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    gap = 2.0 * 0.05 if hole_gap is None else hole_gap
    holes = _place_holes(3, n_holes, r_range, gap, 2 * h, rng)

    def bc_walls(axis, side):
        return BC_T_NEUMANN, 0.0

    return _build(f"cube-spheres-n{n}-b{band:g}", 3, n, holes, band, 0.0, seed + 1000,
                  bc_walls, lambda i: float(i % 2), 0.5)


def holes_refined(dim=2, n=100, n_holes=4, r_range=(0.06, 0.12), delta_h=4.0, ratio=3.0,
                  all_scattered=False, seed=SEED_BASE + 50, hole_gap=0.1):
    """h-refined irregular domain (Section 4.2 in 2D, Section 4.3 in 3D): the
    unit square (cube) minus ``n_holes`` seeded circular (spherical) holes.
    The internodal distance falls linearly from h_r = 1/n (the regular
    lattice) to h_s = h_r/ratio on the hole surfaces over a distance
    h_r*delta_h; the scattered layer has the same width, or covers the whole
    domain when ``all_scattered`` (then the refinement still spans h_r*delta_h).
    Box insulated; holes alternate T_C = 0 / T_H = 1.  ``spacing`` holds h(x_i)."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    holes = _place_holes(dim, n_holes, r_range, hole_gap, 2 * h, rng)
    h_s = h / ratio
    dist = h * delta_h

    def hfun(p):
        g = _min_hole_gap(p, holes, dim)
        return h_s + (h - h_s) * np.clip(g / dist, 0.0, 1.0)

    def bc_walls(axis, side):
        return BC_T_NEUMANN, 0.0

    band = 4.0 if all_scattered else dist
    kind = "allscat" if all_scattered else "hybrid"
    return _build(f"{'square' if dim == 2 else 'cube'}-refined-n{n}-d{delta_h:g}-r{ratio:g}-{kind}", dim, n,
                  holes, band, 0.0, seed + 1000, bc_walls, lambda i: float(i % 2), 0.5, hfun=hfun, h_min=h_s)


def square_all_scattered(n=400, seed=SEED_BASE + 4, jitter=0.0):
    """Unit square filled only with Poisson-disk scattered nodes of spacing 1/n
    (plus the lattice wall nodes); each interior node is then displaced by
    jitter*h*U(unit disk).  Training/test stencils of the learned predictor."""
    ns = _build(f"square-scattered-n{n}", 2, n, np.zeros((0, 3)), 0.0, 1.0, seed,
                lambda a, s: (BC_T_NEUMANN, 0.0), lambda i: 0.0, 0.0)
    return jittered(ns, jitter, seed + 77) if jitter > 0.0 else ns


def jittered(ns, jitter, seed):
    """Copy of a 2D node set with every interior node displaced by
    jitter*h*U(unit disk) (seeded)."""
    rng = np.random.default_rng(seed)
    coords = ns.coords.copy()
    inner = ns.is_boundary == 0
    m = int(inner.sum())
    th = rng.uniform(0, 2 * math.pi, m)
    rr = np.sqrt(rng.uniform(0, 1, m)) * jitter * ns.h
    coords[0, inner] += rr * np.cos(th)
    coords[1, inner] += rr * np.sin(th)
    return NodeSet(f"{ns.name}-j{jitter:g}", ns.dim, ns.h, coords, ns.is_regular.copy(), ns.is_boundary.copy(),
                   ns.normals.copy(), ns.bc.copy(), ns.T_bc.copy(), ns.T_ref, ns.holes, ns.band, ns.spacing)


def scatter_fraction(ns: NodeSet) -> float:
    return ns.n_scattered / ns.N


def square_holes_fraction(target, n=500, seed=SEED_BASE + 1, tol=0.01, iters=30):
    """square_holes with the band width bisected until the scattered fraction is
    within ``tol`` of ``target``; target >= 1 gives the all-scattered set."""
    if target >= 1.0:
        return square_holes(n=n, band=2.0, seed=seed)
    lo, hi = 0.0, 1.0
    best = None
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        ns = square_holes(n=n, band=mid, seed=seed)
        f = scatter_fraction(ns)
        best = ns
        if abs(f - target) <= tol:
            return ns
        if f < target:
            lo = mid
        else:
            hi = mid
    return best


# --------------------------------------------------------------------------
# Smooth test fields (closed-form derivatives)
# --------------------------------------------------------------------------
def field_sincos(coords):
    """u = sin(pi x) cos(pi y) and its exact dx, dy, Laplacian."""
    x, y = coords[0], coords[1]
    u = np.sin(np.pi * x) * np.cos(np.pi * y)
    ux = np.pi * np.cos(np.pi * x) * np.cos(np.pi * y)
    uy = -np.pi * np.sin(np.pi * x) * np.sin(np.pi * y)
    lap = -2.0 * np.pi ** 2 * u
    return u, {"dx": ux, "dy": uy, "lap": lap}


def field_random_smooth(coords, seed=SEED_BASE + 3, q=8):
    """u = sum_q a_q sin(k_q . x + phi_q) with seeded a, k, phi; exact gradient
    and Laplacian."""
    rng = np.random.default_rng(seed)
    dim = coords.shape[0]
    a = rng.normal(size=q)
    kv = rng.uniform(-2 * np.pi, 2 * np.pi, (q, dim))
    ph = rng.uniform(0, 2 * np.pi, q)
    arg = kv @ coords + ph[:, None]
    s, c = np.sin(arg), np.cos(arg)
    u = (a[:, None] * s).sum(0)
    der = {}
    for k, nm in enumerate(["dx", "dy", "dz"][:dim]):
        der[nm] = (a[:, None] * kv[:, k:k + 1] * c).sum(0)
    der["lap"] = -(a[:, None] * (kv ** 2).sum(1)[:, None] * s).sum(0)
    return u, der


def seeded_uniform(shape, seed, lo=-1.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, shape)


# --------------------------------------------------------------------------
# Disk cache for the large sets (generation takes seconds to a minute)
# --------------------------------------------------------------------------
def cached(fn, *args, cache_dir=None, **kw):
    cache_dir = cache_dir or os.environ.get("HSM_NODESET_CACHE",
                                            os.path.join(os.path.dirname(__file__), "..", "build", "nodesets"))
    key = hashlib.sha1(repr((fn.__name__, args, sorted(kw.items()))).encode()).hexdigest()[:16]
    path = os.path.join(cache_dir, f"{fn.__name__}-{key}.npz")
    if os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        spacing = z["spacing"] if "spacing" in z.files and z["spacing"].size else None
        return NodeSet(str(z["name"]), int(z["dim"]), float(z["h"]), z["coords"], z["is_regular"],
                       z["is_boundary"], z["normals"], z["bc"], z["T_bc"], float(z["T_ref"]),
                       z["holes"], float(z["band"]), spacing)
    ns = fn(*args, **kw)
    os.makedirs(cache_dir, exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp.npz"
    np.savez(tmp, name=ns.name, dim=ns.dim, h=ns.h, coords=ns.coords, is_regular=ns.is_regular,
             is_boundary=ns.is_boundary, normals=ns.normals, bc=ns.bc, T_bc=ns.T_bc,
             T_ref=ns.T_ref, holes=ns.holes, band=ns.band,
             spacing=np.zeros(0) if ns.spacing is None else ns.spacing)
    os.replace(tmp, path)
    return ns


def tiled(ns, nx, ny, jitter=None, seed=0):
    """nx x ny copies of a 2D node set side by side, each shifted by a whole
    number of lattice spacings (1 + 2h) so lattice nodes stay on one global
    lattice; ``jitter`` (a callable copy index -> jitter fraction, or None)
    displaces the interior nodes of each copy as ``jittered`` does.  Builds
    million-node workloads from one Poisson-disk fill."""
    n = int(round(1.0 / ns.h))
    step = (n + 2) * ns.h
    parts = []
    for iy in range(ny):
        for ix in range(nx):
            k = iy * nx + ix
            c = jittered(ns, jitter(k), seed + k) if jitter is not None and jitter(k) > 0 else ns
            coords = c.coords.copy()
            coords[0] += ix * step
            coords[1] += iy * step
            parts.append((coords, c))
    cat = lambda f: np.concatenate([f(c) for _, c in parts], -1)
    coords = np.concatenate([p[0] for p in parts], 1)
    return NodeSet(f"{ns.name}-tiled{nx}x{ny}", ns.dim, ns.h, coords, cat(lambda c: c.is_regular),
                   cat(lambda c: c.is_boundary), np.concatenate([c.normals for _, c in parts], 1),
                   cat(lambda c: c.bc), cat(lambda c: c.T_bc), ns.T_ref, ns.holes, ns.band,
                   None if ns.spacing is None else cat(lambda c: c.spacing))
