"""MON and RBF-FD stencil weights, FP64, plain.  Test infrastructure only.

Eq. 1: (L u)(x_c) ~= sum_i w_i u(x_i).  The weights are fixed by requiring Eq. 1
to be exact for a set of basis functions (Section 2), which gives the linear
system M w = l of Section 2.1.  Two bases:

(i)  RBF-FD: polyharmonic spline phi(r) = r^3 (order k = 3, Section 4) on the n
     stencil nodes, augmented with all monomials of total degree <= m.  The
     system is the usual augmented (saddle-point) one

         [ A   P ] [ w      ]   [ L phi(|x - x_i|) at x_c ]
         [ P^T 0 ] [ lambda ] = [ L p_j at x_c            ]

     with A_ij = phi(|x_i - x_j|), P_ij = p_j(x_i - x_c).
(ii) MON: the 2d+1 monomials {1, x_k, x_k^2} (no mixed terms, Section 2
     footnote) on the 2d+1 node regular stencil: P^T w = L p.

Readings where the paper is silent:
* Monomials are taken in offsets from the stencil centre (x - x_c); the
  "centred at the stencil nodes" wording is read as centred at the centre.
* Every system is solved in the scaled variable xi = (x - x_c)/s with
  s = max_i |x_i - x_c|; first-derivative weights are then divided by s and
  Laplacian weights by s^2.  In exact arithmetic this changes nothing (r^3 is
  homogeneous, the monomial space is closed under scaling); it only keeps the
  FP64 solve well conditioned.
* Monomial order (graded lexicographic) does not change the weights.

Right-hand sides, with the centre at xi = 0 and r_i = |xi_i|:
  d/dxi_k  phi(|xi - xi_i|) at 0 = 3 r_i (0 - xi_ik)
  Laplace  phi(|xi - xi_i|) at 0 = phi'' + (d-1) phi'/r = 3 (d+1) r_i
  d/dxi_k  monomial at 0 = 1 for the monomial xi_k, else 0
  Laplace  monomial at 0 = 2 for each xi_k^2, else 0
"""
from __future__ import annotations

import itertools

import numpy as np

OPS_2D = ("dx", "dy", "lap")
OPS_3D = ("dx", "dy", "dz", "lap")


def ops_for(dim):
    return OPS_2D if dim == 2 else OPS_3D


def monomial_exponents(dim, m):
    """All exponent tuples of total degree <= m, graded lexicographic."""
    out = []
    for q in range(m + 1):
        for e in itertools.product(range(q, -1, -1), repeat=dim):
            if sum(e) == q:
                out.append(e)
    return out


def mon_exponents(dim):
    """{1, x_1..x_d, x_1^2..x_d^2}: the 2d+1 MON basis (Section 2 footnote)."""
    out = [tuple([0] * dim)]
    for k in range(dim):
        e = [0] * dim
        e[k] = 1
        out.append(tuple(e))
    for k in range(dim):
        e = [0] * dim
        e[k] = 2
        out.append(tuple(e))
    return out


def eval_monomials(exps, xi):
    """xi [..., dim] -> [..., len(exps)]"""
    cols = []
    for e in exps:
        v = np.ones(xi.shape[:-1])
        for k, a in enumerate(e):
            if a:
                v = v * xi[..., k] ** a
        cols.append(v)
    return np.stack(cols, -1)


def L_monomials_at_center(exps, op, dim):
    """L p_j evaluated at xi = 0."""
    out = np.zeros(len(exps))
    for j, e in enumerate(exps):
        if op == "lap":
            if sum(e) == 2 and max(e) == 2:
                out[j] = 2.0
        else:
            k = "xyz".index(op[1])
            if sum(e) == 1 and e[k] == 1:
                out[j] = 1.0
    return out


def _scaled_offsets(coords, stencil):
    """xi [B, n, dim] and s [B] for stencils [B, n] (column 0 = centre)."""
    x = coords.T[stencil]                       # [B, n, dim]
    off = x - x[:, :1, :]
    s = np.sqrt((off ** 2).sum(-1)).max(1)
    s = np.where(s > 0, s, 1.0)
    return off / s[:, None, None], s


def _unscale(w_xi, s, ops):
    out = {}
    for k, op in enumerate(ops):
        p = 2 if op == "lap" else 1
        out[op] = w_xi[:, :, k] / s[:, None] ** p
    return out


def rbffd_system(xi, m, ops):
    """Augmented PHS r^3 system for scaled offsets xi [B, n, dim].
    Returns M [B, K, K] and RHS [B, K, n_ops]."""
    B, n, dim = xi.shape
    exps = monomial_exponents(dim, m)
    Mp = len(exps)
    K = n + Mp
    diff = xi[:, :, None, :] - xi[:, None, :, :]
    r = np.sqrt((diff ** 2).sum(-1))
    A = r ** 3
    P = eval_monomials(exps, xi)                # [B, n, Mp]
    M = np.zeros((B, K, K))
    M[:, :n, :n] = A
    M[:, :n, n:] = P
    M[:, n:, :n] = np.transpose(P, (0, 2, 1))
    rc = np.sqrt((xi ** 2).sum(-1))             # [B, n]
    rhs = np.zeros((B, K, len(ops)))
    for k, op in enumerate(ops):
        if op == "lap":
            rhs[:, :n, k] = 3.0 * (dim + 1) * rc
        else:
            a = "xyz".index(op[1])
            rhs[:, :n, k] = 3.0 * rc * (0.0 - xi[:, :, a])
        rhs[:, n:, k] = L_monomials_at_center(exps, op, dim)[None, :]
    return M, rhs


# A stencil is unisolvent for the monomials of degree <= m when P has full
# column rank; numerically, when its smallest singular value exceeds this
# fraction of its largest (P of the scaled offsets has entries of order one).
UNISOLVENT_RTOL = 1e-10


def unisolvent(xi, m):
    """[B] bool: the monomials of degree <= m are unisolvent on the scaled
    stencil offsets xi [B, n, dim] (P [B, n, Mp] of full column rank)."""
    P = eval_monomials(monomial_exponents(xi.shape[-1], m), xi)
    sv = np.linalg.svd(P, compute_uv=False)
    return sv[:, -1] > UNISOLVENT_RTOL * sv[:, 0]


def rbffd_weights_degree(coords, stencil, m, ops=None):
    """RBF-FD weights for stencils [B, n] and the monomial degree each used.

    Reading (the paper requires a stencil whose system is solvable at every
    node, Section 2): a stencil on which the monomials of degree <= m are not
    unisolvent -- e.g. a 3D wall node next to a box edge whose stencil spans
    three lattice layers across the edge, where a cubic vanishes on every
    node -- takes the largest degree m' < m (m' >= 1) that is unisolvent on
    the same n nodes.  Returns ({op: w [B, n]}, m_used [B])."""
    dim = coords.shape[0]
    ops = ops or ops_for(dim)
    stencil = np.asarray(stencil)
    n = stencil.shape[1] if stencil.ndim == 2 else 0
    if len(stencil) == 0:
        return {op: np.zeros((0, n)) for op in ops}, np.zeros(0, dtype=np.int64)
    xi, s = _scaled_offsets(coords, stencil)
    m_used = np.full(len(stencil), m, dtype=np.int64)
    todo = ~unisolvent(xi, m)
    for mm in range(m - 1, 0, -1):
        if not todo.any():
            break
        m_used[todo] = mm
        sub = np.flatnonzero(todo)
        todo[sub] = ~unisolvent(xi[sub], mm)
    sol = np.zeros((len(stencil), n, len(ops)))
    for mm in np.unique(m_used):
        sel = np.flatnonzero(m_used == mm)
        M, rhs = rbffd_system(xi[sel], int(mm), ops)
        sol[sel] = np.linalg.solve(M, rhs)[:, :n, :]
    return _unscale(sol, s, ops), m_used


def rbffd_weights(coords, stencil, m, ops=None):
    """RBF-FD weights for stencils [B, n].  Returns {op: w [B, n]}."""
    return rbffd_weights_degree(coords, stencil, m, ops)[0]


def mon_system(xi, ops):
    B, n, dim = xi.shape
    exps = mon_exponents(dim)
    P = eval_monomials(exps, xi)                # [B, n, 2d+1]
    Mt = np.transpose(P, (0, 2, 1))             # rows = basis functions
    rhs = np.stack([L_monomials_at_center(exps, op, dim) for op in ops], -1)
    rhs = np.broadcast_to(rhs, (B,) + rhs.shape).copy()
    return Mt, rhs


def mon_weights(coords, stencil, ops=None):
    """MON weights for regular stencils [B, 2d+1]: P^T w = L p."""
    dim = coords.shape[0]
    ops = ops or ops_for(dim)
    stencil = np.asarray(stencil)
    if len(stencil) == 0:
        return {op: np.zeros((0, stencil.shape[1])) for op in ops}
    xi, s = _scaled_offsets(coords, stencil)
    Mt, rhs = mon_system(xi, ops)
    sol = np.linalg.solve(Mt, rhs)
    return _unscale(sol, s, ops)


def all_weights(coords, st, m, ops=None):
    """Weights for the stencils returned by ``stencils.build_stencils``."""
    dim = coords.shape[0]
    ops = ops or ops_for(dim)
    w_rbf, m_used = rbffd_weights_degree(coords, st["rbf_idx"], m, ops)
    return dict(mon=mon_weights(coords, st["mon_idx"], ops), rbf=w_rbf, rbf_m=m_used)


def stencil_size(dim, m):
    """n = 2 * C(m+d, m) (Section 1, the standard recommendation)."""
    from math import comb

    return 2 * comb(m + dim, m)


def condition_numbers(coords, st, m):
    """2-norm condition numbers kappa(M) = ||M|| ||M^-1|| of every stencil's
    weight system (Section 2.1, "Computational stability"): the scaled MON
    matrix P^T of a regular node, the scaled augmented RBF-FD matrix of a
    scattered one.  Scaling by s = max |x_i - x_c| as for the weights.
    Returns {"mon": [N_mon], "rbf": [N_rbf]}."""
    dim = coords.shape[0]
    ops = ops_for(dim)
    out = {}
    if len(st["mon_idx"]):
        xi, _ = _scaled_offsets(coords, np.asarray(st["mon_idx"]))
        Mt, _ = mon_system(xi, ops)
        out["mon"] = np.linalg.cond(Mt, 2)
    else:
        out["mon"] = np.zeros(0)
    if len(st["rbf_idx"]):
        xi, _ = _scaled_offsets(coords, np.asarray(st["rbf_idx"]))
        M, _ = rbffd_system(xi, m, ops)
        out["rbf"] = np.linalg.cond(M, 2)
    else:
        out["rbf"] = np.zeros(0)
    return out
