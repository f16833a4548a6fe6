"""Pins for the oracle's stencil selection (Section 2: n neighbouring nodes)."""
import json
import os

import numpy as np

from oracle import stencils as ost
from paper_2303_01760_gb300 import nodesets

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _lattice_coords(L, h=1.0):
    j, i = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    return np.stack([i.ravel() * h, j.ravel() * h], 0).astype(np.float64)


def test_knn_hand_worked_ties():
    g = json.load(open(os.path.join(GOLD, "knn_tie_5x5.json")))
    coords = _lattice_coords(g["lattice"])
    got = ost.knn_bruteforce(coords, [g["center"]], g["n"])[0]
    assert got.tolist() == g["expected"]
    got_kd = ost.knn_kdtree(coords, [g["center"]], g["n"])[0]
    assert got_kd.tolist() == g["expected"]


def test_knn_kdtree_equals_bruteforce():
    ns = nodesets.square_wall_band(n=24)
    rng = np.random.default_rng(5)
    centers = rng.choice(ns.N, 200, replace=False)
    for n in (12, 30):
        a = ost.knn_bruteforce(ns.coords, centers, n)
        b = ost.knn_kdtree(ns.coords, centers, n)
        assert np.array_equal(a, b)
        assert np.all(a[:, 0] == centers)


def test_knn_3d_kdtree_equals_bruteforce():
    rng = np.random.default_rng(6)
    # a lattice plus jittered points: many exact ties
    g = np.stack(np.meshgrid(*[np.arange(6)] * 3, indexing="ij"), 0).reshape(3, -1) / 5.0
    coords = np.concatenate([g, rng.uniform(0, 1, (3, 100))], 1)
    centers = np.arange(0, coords.shape[1], 3)
    for n in (20, 40):
        assert np.array_equal(ost.knn_bruteforce(coords, centers, n), ost.knn_kdtree(coords, centers, n))


def test_knn_is_sorted_by_distance_then_id():
    ns = nodesets.square_wall_band(n=16)
    idx = ost.knn_bruteforce(ns.coords, np.arange(ns.N), 12)
    for c, row in enumerate(idx):
        d2 = ost.sq_dist(ns.coords, c, row)
        key = list(zip(d2.tolist(), row.tolist()))
        assert key == sorted(key)
        # nothing outside the stencil is strictly closer than its last member
        all_d2 = ost.sq_dist(ns.coords, c)
        outside = np.setdiff1d(np.arange(ns.N), row)
        assert np.all((all_d2[outside] > d2[-1]) | ((all_d2[outside] == d2[-1]) & (outside > row[-1])))


def test_mon_stencil_order_and_demotion():
    ns = nodesets.square_wall_band(n=40)
    mon_nodes, mon_idx, demoted = ost.mon_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h)
    h = ns.h
    off = ns.coords[:, mon_idx] - ns.coords[:, mon_idx[:, :1]]
    expect = np.array([[0, -h, h, 0, 0], [0, 0, 0, -h, h]])
    assert np.allclose(off, expect[:, None, :], atol=1e-12)
    # the 0.1-wide wall band removes lattice nodes, so the outermost regular ring is demoted
    assert len(demoted) > 0
    assert len(mon_nodes) + len(demoted) == int(ns.is_regular.sum())
    for c in demoted:
        q = np.rint(ns.coords[:, c] / h).astype(int)
        assert np.any(q == 4) or np.any(q == 36)


def test_paper_regular_dvd_node_count():
    """Table 1: N = 64 005 on the regular discretisation, a 253^2 lattice
    without its corners; the generator's lattice rule reproduces it."""
    g = json.load(open(os.path.join(GOLD, "paper_values.json")))["dvd_regular_N"]
    n = g["lattice_points_per_axis"] - 1
    ns = nodesets.square_wall_band(n=n, wall_band=0.0)
    assert ns.N == g["value"]
    assert ns.n_scattered == int(ns.is_boundary.sum())


def test_boundary_search_point_moves_by_the_local_spacing():
    """Hand-worked: a wall node at (0, 0.5) with outward normal (-1, 0) and
    interior nodes on a 0.1 grid.  With spacing 0.1 the search point is
    (0.1, 0.5) and the nearest interior node is the one there; with a local
    spacing of 0.3 (an h-refined set) the search point is (0.3, 0.5)."""
    xs = np.arange(1, 6) * 0.1
    ys = np.arange(3, 8) * 0.1
    gx, gy = np.meshgrid(xs, ys, indexing="xy")
    coords = np.concatenate([[[0.0], [0.5]], np.stack([gx.ravel(), gy.ravel()])], 1)
    normals = np.zeros_like(coords)
    normals[0, 0] = -1.0
    is_bnd = np.zeros(coords.shape[1], dtype=np.uint8)
    is_bnd[0] = 1
    interior = is_bnd == 0
    at = lambda x, y: int(np.flatnonzero(np.isclose(coords[0], x) & np.isclose(coords[1], y))[0])
    got = ost.boundary_bruteforce(coords, normals, 0.1, [0], 2, interior)[0]
    assert got.tolist() == [0, at(0.1, 0.5)]
    spacing = np.full(coords.shape[1], 0.1)
    assert ost.boundary_bruteforce(coords, normals, spacing, [0], 2, interior)[0].tolist() == got.tolist()
    spacing[0] = 0.3
    assert ost.boundary_bruteforce(coords, normals, spacing, [0], 2, interior)[0].tolist() == [0, at(0.3, 0.5)]
    assert ost.boundary_kdtree(coords, normals, spacing, [0], 2, interior)[0].tolist() == [0, at(0.3, 0.5)]
    # the whole-set builder takes the spacing array the same way
    st = ost.build_stencils(coords, np.zeros(coords.shape[1], np.uint8), is_bnd, 0.1, 2, normals=normals,
                            spacing=spacing)
    r = int(np.flatnonzero(st["rbf_nodes"] == 0)[0])
    assert st["rbf_idx"][r].tolist() == [0, at(0.3, 0.5)]


def test_refined_boundary_stencils_are_more_local():
    """On an h-refined set (spacing h_r/3 at the holes) hole-node stencils
    searched one LOCAL spacing inside keep each node's nearest interior
    neighbour and reach less far than those searched a whole lattice spacing
    inside."""
    ns = nodesets.holes_refined(n=30, n_holes=2, r_range=(0.1, 0.15), delta_h=4.0, seed=nodesets.SEED_BASE + 60)
    hole = np.flatnonzero((ns.is_boundary == 1) & (ns.bc == nodesets.BC_T_DIRICHLET))
    interior = ns.is_boundary == 0
    reach = {}
    for name, hh in (("local", ns.spacing), ("lattice", ns.h)):
        st = ost.boundary_bruteforce(ns.coords, ns.normals, hh, hole, 12, interior)
        far = []
        for r, c in enumerate(hole):
            far.append(np.sqrt(ost.sq_dist(ns.coords, int(c), st[r, 1:])).max() / ns.spacing[c])
            if name == "local":
                nearest = int(np.argmin(np.where(interior, ost.sq_dist(ns.coords, int(c)), np.inf)))
                assert nearest in st[r]
        reach[name] = np.median(far)
    assert reach["local"] < 0.9 * reach["lattice"]


def test_subset_build_equals_full_build_on_those_nodes():
    """Stencils built for a subset of centres (as the full-size sampled parity
    tests do) are the full build's stencils of those nodes."""
    ns = nodesets.square_holes(n=60, n_holes=3, r_range=(0.08, 0.12), band=0.08, seed=nodesets.SEED_BASE + 31)
    full = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, 12, normals=ns.normals)
    rng = np.random.default_rng(3)
    centers = np.unique(rng.choice(ns.N, 400, replace=False))
    sub = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, 12, centers=centers,
                             normals=ns.normals)
    for grp in ("mon", "rbf"):
        rows = {int(c): r.tolist() for c, r in zip(full[grp + "_nodes"], full[grp + "_idx"])}
        assert set(sub[grp + "_nodes"].tolist()) == set(rows) & set(centers.tolist())
        for c, r in zip(sub[grp + "_nodes"], sub[grp + "_idx"]):
            assert r.tolist() == rows[int(c)]
    assert set(sub["demoted"].tolist()) == set(full["demoted"].tolist()) & set(centers.tolist())
