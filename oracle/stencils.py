"""Stencil selection, FP64, plain.  Test infrastructure only (see package doc).

Section 2: the operator at x_c is approximated over "a set of n neighbouring
nodes".  Readings taken where the paper is silent:

* Scattered stencil = the n nodes with the smallest key (d2, id), where
  d2 = ((dx*dx) + (dy*dy)) + (dz*dz) in float64, evaluated exactly in that
  order with dx = x_i - x_c, and id the node index.  The centre (d2 = 0) comes
  first.  Ties go to the lower node id.
* Regular (MON) stencil = {c, c-e1, c+e1, c-e2, c+e2[, c-e3, c+e3]} looked up
  through integer lattice coordinates round(x/h).  A node is on the lattice
  when every |x_k/h - round(x_k/h)| <= 1e-6; if two nodes share a lattice point
  the lower id owns it.
* A boundary node's stencil is the node itself followed by the n-1 interior
  (non-boundary) nodes nearest to the point q = x_c - h n_c one lattice
  spacing inside along the outward normal n_c, ordered by the same key with d2
  measured from q (q_k = x_ck - (h * n_ck), no fused multiply-add).  On an
  h-refined node set (Sections 4.2 and 4.3: the internodal distance h(x)
  falls towards the irregular boundary) h is the local spacing h(x_c), so the
  search point stays one local spacing inside.  Boundary
  stencils serve only the normal-derivative rows of the Neumann conditions.
  Keeping other boundary nodes out of them makes each such row hold exactly
  after an explicit update (with boundary neighbours the explicit closure
  couples the walls and its error grows from step to step); centring the
  search inside keeps several node layers in the stencil, without which the
  monomial part is singular on a 3D lattice wall.
* A node uses MON only when it is flagged regular, is not a boundary node and
  all 2d lattice neighbours exist; any other regular-flagged node is demoted to
  RBF-FD (Section 2 notes that MON is only stable on regular nodes).
"""
from __future__ import annotations

import numpy as np

LATTICE_TOL = 1e-6


def sq_dist(coords, c, ids=None):
    """float64 d2 from node c to nodes ``ids`` (all nodes when None), summed in
    coordinate order with no fused multiply-add."""
    dim = coords.shape[0]
    if ids is None:
        ids = slice(None)
    d2 = None
    for k in range(dim):
        dk = coords[k, ids] - coords[k, c]
        t = dk * dk
        d2 = t if d2 is None else d2 + t
    return d2


def sq_dist_point(coords, q, ids=None):
    """float64 d2 from the point q [dim] to nodes ``ids``, as ``sq_dist``."""
    dim = coords.shape[0]
    if ids is None:
        ids = slice(None)
    d2 = None
    for k in range(dim):
        dk = coords[k, ids] - q[k]
        t = dk * dk
        d2 = t if d2 is None else d2 + t
    return d2


def knn_bruteforce(coords, centers, n):
    """Definition: for each centre, all N distances, order by (d2, id), keep n."""
    N = coords.shape[1]
    ids = np.arange(N)
    out = np.empty((len(centers), n), dtype=np.int64)
    for r, c in enumerate(centers):
        d2 = sq_dist(coords, int(c))
        order = np.lexsort((ids, d2))
        out[r] = order[:n]
    return out


def inward_point(coords, normals, h, c):
    """q = x_c - (h * n_c), evaluated per coordinate without fused multiply-add;
    ``h`` is a scalar or a per-node spacing array (then h = h[c])."""
    hc = float(h[c]) if np.ndim(h) else h
    return np.array([coords[k, c] - (hc * normals[k, c]) for k in range(coords.shape[0])])


def boundary_bruteforce(coords, normals, h, centers, n, interior):
    """Definition for boundary nodes: [c] + the n-1 interior nodes of smallest
    (d2 from q, id), q = x_c - h n_c."""
    N = coords.shape[1]
    ids = np.arange(N)
    out = np.empty((len(centers), n), dtype=np.int64)
    for r, c in enumerate(centers):
        q = inward_point(coords, normals, h, int(c))
        d2 = np.where(interior, sq_dist_point(coords, q), np.inf)
        order = np.lexsort((ids, d2))
        out[r, 0] = c
        out[r, 1:] = order[:n - 1]
    return out


def boundary_kdtree(coords, normals, h, centers, n, interior, margin=8):
    """Same result as ``boundary_bruteforce`` via a k-d tree over the interior
    nodes, with the completeness guard of ``knn_kdtree``."""
    from scipy.spatial import cKDTree

    pool = np.flatnonzero(interior)
    tree = cKDTree(coords.T[pool])
    out = np.empty((len(centers), n), dtype=np.int64)
    for r, c in enumerate(centers):
        q = inward_point(coords, normals, h, int(c))
        kk = n - 1 + margin
        while True:
            kq = min(kk, len(pool))
            dist, idx = tree.query(q, k=kq)
            dist, idx = np.atleast_1d(dist), pool[np.atleast_1d(idx)]
            if kq == len(pool) or dist[-1] > dist[n - 2] * (1.0 + 1e-9) + 1e-300:
                break
            kk *= 2
        d2 = sq_dist_point(coords, q, idx)
        order = np.lexsort((idx, d2))
        out[r, 0] = c
        out[r, 1:] = idx[order[:n - 1]]
    return out


def knn_kdtree(coords, centers, n, margin=8):
    """Same result as ``knn_bruteforce`` for large N.  A k-d tree proposes the
    nearest n+margin candidates; the candidate set is provably complete when the
    last candidate is strictly farther than the n-th (with a relative guard
    against the tree's own rounding), otherwise the query is widened.  The final
    order is taken with the exact (d2, id) key."""
    from scipy.spatial import cKDTree

    pts = coords.T
    tree = cKDTree(pts)
    centers = np.asarray(centers, dtype=np.int64)
    out = np.empty((len(centers), n), dtype=np.int64)
    todo = np.arange(len(centers))
    kk = n + margin
    while len(todo):
        kq = min(kk, coords.shape[1])
        dist, idx = tree.query(pts[centers[todo]], k=kq)
        dist = np.atleast_2d(dist)
        idx = np.atleast_2d(idx)
        complete = (kq == coords.shape[1]) | (dist[:, -1] > dist[:, n - 1] * (1.0 + 1e-9) + 1e-300)
        for r in np.flatnonzero(complete):
            c = int(centers[todo[r]])
            cand = idx[r]
            d2 = sq_dist(coords, c, cand)
            order = np.lexsort((cand, d2))
            out[todo[r]] = cand[order[:n]]
        todo = todo[~complete]
        kk *= 2
    return out


def lattice_map(coords, h):
    """Dict lattice ijk tuple -> lowest node id lying on that lattice point."""
    dim, N = coords.shape
    q = coords / h
    r = np.rint(q)
    on = np.all(np.abs(q - r) <= LATTICE_TOL, axis=0)
    m = {}
    ri = r.astype(np.int64)
    for i in np.flatnonzero(on):
        key = tuple(int(v) for v in ri[:, i])
        if key not in m:
            m[key] = int(i)
    return m, ri, on


def mon_stencils(coords, is_regular, is_boundary, h, only=None):
    """Regular stencils.  Returns (nodes, idx[len(nodes), 2d+1]) for the nodes
    that keep MON, and the array of demoted node ids; with ``only`` (node ids)
    just for those of them that are flagged regular."""
    dim, N = coords.shape
    m, ri, on = lattice_map(coords, h)
    nodes, rows, demoted = [], [], []
    cand = np.flatnonzero(is_regular) if only is None else np.asarray(only)[np.asarray(is_regular)[only] != 0]
    for c in cand:
        c = int(c)
        if is_boundary[c] or not on[c] or m.get(tuple(int(v) for v in ri[:, c])) != c:
            demoted.append(c)
            continue
        row = [c]
        ok = True
        for k in range(dim):
            for sgn in (-1, 1):
                key = list(int(v) for v in ri[:, c])
                key[k] += sgn
                j = m.get(tuple(key))
                if j is None:
                    ok = False
                    break
                row.append(j)
            if not ok:
                break
        if ok:
            nodes.append(c)
            rows.append(row)
        else:
            demoted.append(c)
    idx = np.array(rows, dtype=np.int64).reshape(len(rows), 2 * dim + 1)
    return np.array(nodes, dtype=np.int64), idx, np.array(demoted, dtype=np.int64)


def build_stencils(coords, is_regular, is_boundary, h, n, centers=None, use_kdtree=None, normals=None,
                   spacing=None):
    """All stencils of a node set (or of the subset ``centers``).  ``spacing``
    (optional, [N]) is the local internodal distance of an h-refined set; it
    replaces h in the search point of boundary stencils.

    Returns dict with
      mon_nodes, mon_idx   nodes that use MON and their 2d+1 stencil
      rbf_nodes, rbf_idx   nodes that use RBF-FD (scattered + demoted) and their
                           n-node stencil
      demoted              regular-flagged nodes demoted to RBF-FD
    """
    dim, N = coords.shape
    mon_nodes, mon_idx, demoted = mon_stencils(coords, is_regular, is_boundary, h,
                                               only=None if centers is None else np.asarray(centers, dtype=np.int64))
    kind = np.ones(N, dtype=np.int8)  # 1 = RBF-FD
    kind[mon_nodes] = 0
    if centers is not None:
        centers = np.asarray(centers, dtype=np.int64)
        sel = kind[centers] == 0
        keep = np.isin(mon_nodes, centers)
        mon_nodes, mon_idx = mon_nodes[keep], mon_idx[keep]
        rbf_nodes = centers[~sel]
    else:
        rbf_nodes = np.flatnonzero(kind == 1)
    if use_kdtree is None:
        use_kdtree = N * len(rbf_nodes) > 2e7
    knn = knn_kdtree if use_kdtree else knn_bruteforce
    rbf_idx = np.zeros((len(rbf_nodes), n), dtype=np.int64)
    on_bnd = np.asarray(is_boundary)[rbf_nodes] != 0
    if np.any(~on_bnd):
        rbf_idx[~on_bnd] = knn(coords, rbf_nodes[~on_bnd], n)
    if np.any(on_bnd):
        if normals is None:
            raise ValueError("boundary nodes need their normals")
        bk = boundary_kdtree if use_kdtree else boundary_bruteforce
        hb = h if spacing is None else np.asarray(spacing, dtype=np.float64)
        rbf_idx[on_bnd] = bk(coords, normals, hb, rbf_nodes[on_bnd], n, np.asarray(is_boundary) == 0)
    return dict(mon_nodes=mon_nodes, mon_idx=mon_idx, rbf_nodes=rbf_nodes, rbf_idx=rbf_idx,
                demoted=demoted)
