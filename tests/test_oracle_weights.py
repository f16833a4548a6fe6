"""Pins for the oracle's MON and RBF-FD weights (Eq. 1, Section 2 and 2.1)."""
import json
import os
from math import comb

import numpy as np
import pytest

from oracle import stencils as ost
from oracle import weights as ow
from oracle import apply as oap
from paper_2303_01760_gb300 import nodesets

GOLD = os.path.join(os.path.dirname(__file__), "golden")
PAPER = json.load(open(os.path.join(GOLD, "paper_values.json")))


def test_stencil_sizes_match_paper():
    assert ow.stencil_size(2, 2) == PAPER["stencil_n_2d_m2"]["value"]
    assert len(ow.mon_exponents(2)) == PAPER["mon_n_2d"]["value"]
    assert len(ow.mon_exponents(3)) == PAPER["mon_n_3d"]["value"]
    assert len(ow.monomial_exponents(2, 2)) == comb(4, 2)
    assert len(ow.monomial_exponents(3, 3)) == comb(6, 3)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("h", [1.0 / 40, 0.002, 1.0 / 7])
def test_mon_closed_form_classical_fd(dim, h):
    """Section 2 footnote: on the symmetric 2d+1 node lattice stencil the MON
    weights are the classical central differences: Laplacian (-2d, 1..1)/h^2,
    d/dx_k = -+1/(2h) on c -+ e_k."""
    c = np.full(dim, 3.0) * h
    pts = [c]
    for k in range(dim):
        for s in (-1, 1):
            p = c.copy()
            p[k] += s * h
            pts.append(p)
    coords = np.array(pts).T
    W = ow.mon_weights(coords, np.arange(2 * dim + 1)[None, :])
    lap = np.r_[-2.0 * dim, np.ones(2 * dim)] / h ** 2
    assert np.allclose(W["lap"][0], lap, rtol=0, atol=1e-12 * abs(lap).max())
    for k, op in enumerate(["dx", "dy", "dz"][:dim]):
        e = np.zeros(2 * dim + 1)
        e[1 + 2 * k] = -0.5 / h
        e[2 + 2 * k] = 0.5 / h
        assert np.allclose(W[op][0], e, rtol=0, atol=1e-12 / h)


def _stencil_cloud(dim, n, seed, jitter=0.35):
    """A quasi-uniform cloud (jittered lattice) and the n-node stencil of its
    most central node."""
    rng = np.random.default_rng(seed)
    L = 7 if dim == 2 else 5
    g = np.stack(np.meshgrid(*[np.arange(L)] * dim, indexing="ij"), 0).reshape(dim, -1).astype(float)
    g += rng.uniform(-jitter, jitter, g.shape)
    coords = g * 0.01 + 0.3
    c = int(np.argmin(((g - (L - 1) / 2) ** 2).sum(0)))
    st = ost.knn_bruteforce(coords, [c], n)
    return coords, st


def _rbf_space_function(coords, st, m, seed):
    """u(x) = sum_i c_i |x - x_i|^3 + q(x), with c in the null space of P^T
    (so u lies in the RBF-FD interpolation space) and q a random polynomial of
    degree <= m.  Returned as an mpmath-evaluable function."""
    import mpmath as mp

    dim = coords.shape[0]
    rng = np.random.default_rng(seed)
    X = coords[:, st[0]].T
    xc = X[0]
    exps = ow.monomial_exponents(dim, m)
    P = np.array([[np.prod((x - xc) ** np.array(e)) for e in exps] for x in X])
    _, _, vt = np.linalg.svd(P.T)
    Z = vt[len(exps):].T                        # basis of null(P^T)
    cvec = Z @ rng.normal(size=Z.shape[1])
    # normalise both parts to O(1) values on the stencil so neither hides the other
    r = np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    cvec /= np.abs((r ** 3) @ cvec).max()
    s = np.sqrt(((X - xc) ** 2).sum(1)).max()
    qcoef = rng.normal(size=len(exps)) / np.array([s ** sum(e) for e in exps])
    Xm = [[mp.mpf(float(v)) for v in x] for x in X]
    xcm = [mp.mpf(float(v)) for v in xc]

    def u(*x):
        s = mp.mpf(0)
        for ci, xi in zip(cvec, Xm):
            r = mp.sqrt(sum((a - b) ** 2 for a, b in zip(x, xi)))
            s += mp.mpf(float(ci)) * r ** 3
        for qc, e in zip(qcoef, exps):
            t = mp.mpf(float(qc))
            for a, b, k in zip(x, xcm, e):
                t *= (a - b) ** k
            s += t
        return s

    return u, X, xc


@pytest.mark.parametrize("dim,m", [(2, 2), (2, 4), (3, 2), (3, 3)])
def test_rbffd_exact_on_rbf_space_numerical_derivatives(dim, m):
    """Eq. 1 is enforced for the PHS + monomial basis (Section 2), so it must be
    exact for every function of the augmented space.  The exact operator value
    is taken here by high-precision numerical differentiation of the function
    itself, independent of the oracle's closed-form right-hand sides."""
    import mpmath as mp

    mp.mp.dps = 40
    n = ow.stencil_size(dim, m)
    coords, st = _stencil_cloud(dim, n, seed=10 * dim + m)
    W = ow.rbffd_weights(coords, st, m)
    u, X, xc = _rbf_space_function(coords, st, m, seed=3)
    uvals = np.array([float(u(*[mp.mpf(float(v)) for v in x])) for x in X])
    xcm = [mp.mpf(float(v)) for v in xc]
    for k, op in enumerate(ow.ops_for(dim)):
        if op == "lap":
            ref = mp.mpf(0)
            for a in range(dim):
                order = [0] * dim
                order[a] = 2
                ref += mp.diff(u, xcm, tuple(order))
        else:
            order = [0] * dim
            order["xyz".index(op[1])] = 1
            ref = mp.diff(u, xcm, tuple(order))
        ref = float(ref)
        got = float(np.dot(W[op][0], uvals))
        scale = np.abs(W[op][0] * uvals).sum()
        assert abs(got - ref) <= 1e-9 * scale, (op, got, ref)


@pytest.mark.parametrize("dim,m", [(2, 2), (2, 4), (3, 2), (3, 3)])
def test_rbffd_polynomial_reproduction(dim, m):
    n = ow.stencil_size(dim, m)
    coords, st = _stencil_cloud(dim, n, seed=7 + dim + m)
    W = ow.rbffd_weights(coords, st, m)
    X = coords[:, st[0]].T
    xc = X[0]
    for e in ow.monomial_exponents(dim, m):
        # monomials in absolute coordinates about an arbitrary origin
        vals = np.prod((X - xc + 0.25 * 0.01) ** np.array(e), axis=1)
        for op in ow.ops_for(dim):
            # exact derivative of prod (x_k - xc_k + 0.0025)^e_k at x_c
            t = np.full(dim, 0.0025)
            if op == "lap":
                ref = 0.0
                for a in range(dim):
                    if e[a] >= 2:
                        f = e[a] * (e[a] - 1) * t[a] ** (e[a] - 2)
                        ref += f * np.prod([t[b] ** e[b] for b in range(dim) if b != a])
            else:
                a = "xyz".index(op[1])
                ref = 0.0 if e[a] == 0 else e[a] * t[a] ** (e[a] - 1) * np.prod(
                    [t[b] ** e[b] for b in range(dim) if b != a])
            got = np.dot(W[op][0], vals)
            assert abs(got - ref) <= 1e-9 * (np.abs(W[op][0] * vals).sum() + abs(ref) + 1e-30)
        # derivative weights sum to zero (constants are reproduced)
    for op in ow.ops_for(dim):
        assert abs(W[op][0].sum()) <= 1e-10 * np.abs(W[op][0]).sum()


def test_rbffd_solve_accuracy_against_50_digit_solve():
    """Bounds the FP64 solve error of the oracle itself (Section 2.1 system)."""
    import mpmath as mp

    mp.mp.dps = 50
    for dim, m in [(2, 2), (2, 4), (3, 3)]:
        n = ow.stencil_size(dim, m)
        coords, st = _stencil_cloud(dim, n, seed=21 + m)
        xi, s = ow._scaled_offsets(coords, st)
        M, rhs = ow.rbffd_system(xi, m, ow.ops_for(dim))
        sol = np.linalg.solve(M[0], rhs[0])
        Mm = mp.matrix(M[0].tolist())
        for k in range(rhs.shape[2]):
            ex = mp.lu_solve(Mm, mp.matrix(rhs[0, :, k].tolist()))
            ex = np.array([float(v) for v in ex])[:n]
            assert np.abs(sol[:n, k] - ex).max() <= 1e-11 * np.abs(ex).max()


def test_rbffd_translation_and_scale_covariance():
    coords, st = _stencil_cloud(2, 12, seed=4)
    W1 = ow.rbffd_weights(coords, st, 2)
    W2 = ow.rbffd_weights(coords * 3.0 + 0.7, st, 2)
    assert np.allclose(W2["dx"], W1["dx"] / 3.0, rtol=1e-10, atol=0)
    assert np.allclose(W2["lap"], W1["lap"] / 9.0, rtol=1e-10, atol=0)


def _conv_errors(kind, ns_list, m=2):
    errs = {op: [] for op in ("dx", "dy", "lap")}
    hs = []
    for ns in ns_list:
        st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h,
                                ow.stencil_size(2, m), normals=ns.normals)
        W = ow.all_weights(ns.coords, st, m)
        u, der = nodesets.field_sincos(ns.coords)
        out = oap.apply_all(ns.N, st, W, u, ("dx", "dy", "lap"))
        x = ns.coords
        inner = (np.minimum(x, 1 - x).min(0) > 0.2)
        if kind == "mon":
            sel = np.zeros(ns.N, bool)
            sel[st["mon_nodes"]] = True
        else:
            sel = np.zeros(ns.N, bool)
            sel[st["rbf_nodes"]] = True
        sel &= inner
        for op in errs:
            errs[op].append(np.abs(out[op][sel] - der[op][sel]).max())
        hs.append(ns.h)
    return np.array(hs), {k: np.array(v) for k, v in errs.items()}


def test_convergence_mon_on_lattice():
    """Smooth u = sin(pi x) cos(pi y): MON (central differences) converge at
    second order for first and second derivatives."""
    hs, e = _conv_errors("mon", [nodesets.square_wall_band(n=n, wall_band=0.0) for n in (20, 40, 80)])
    for op in e:
        slope = np.polyfit(np.log(hs), np.log(e[op]), 1)[0]
        assert slope > 1.7, (op, slope, e[op])


@pytest.mark.slow
def test_convergence_rbffd_scattered():
    """RBF-FD with m=2 on Poisson-disk nodes: first derivatives converge at
    about order m = 2, the Laplacian at about m - 1 = 1."""
    sets = [nodesets.square_wall_band(n=n, wall_band=1.0, seed=nodesets.SEED_BASE + 50 + n)
            for n in (20, 40, 80)]
    hs, e = _conv_errors("rbf", sets)
    sl = {op: np.polyfit(np.log(hs), np.log(e[op]), 1)[0] for op in e}
    assert sl["dx"] > 1.5 and sl["dy"] > 1.5, sl
    assert sl["lap"] > 0.7, sl


def test_convergence_on_h_refined_sets():
    """h-refined sets (Section 4.2: spacing h_r/3 at the holes, delta_h = 4)
    with boundary stencils searched one local spacing inside: the maximum
    error of the hybrid operators on u = sin(pi x) cos(pi y) over interior
    nodes falls with h_r at about the method's order (m = 2: 2 for the first
    derivatives, 1 for the Laplacian).  Measured least-squares slopes over
    h_r = 1/50, 1/100, 1/200: 2.0 (dx), 1.8 (dy), 1.1 (Laplacian); the bounds
    leave room for the randomness of the node sets."""
    hs, errs = [], {op: [] for op in ("dx", "dy", "lap")}
    for n in (50, 100, 200):
        ns = nodesets.holes_refined(n=n, n_holes=2, r_range=(0.15, 0.2), delta_h=4.0, seed=nodesets.SEED_BASE + 62)
        st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, 12, normals=ns.normals,
                                spacing=ns.spacing)
        W = ow.all_weights(ns.coords, st, 2)
        u, ex = nodesets.field_sincos(ns.coords)
        out = oap.apply_all(ns.N, st, W, u, ("dx", "dy", "lap"))
        inner = ns.is_boundary == 0
        hs.append(ns.h)
        for op in errs:
            errs[op].append(np.abs(out[op][inner] - ex[op][inner]).max())
    slope = {op: np.polyfit(np.log(hs), np.log(errs[op]), 1)[0] for op in errs}
    assert slope["dx"] >= 1.5 and slope["dy"] >= 1.5, slope
    assert slope["lap"] >= 0.8, slope


def test_reduced_degree_on_a_stencil_where_quadratics_are_not_unisolvent():
    """Twelve nodes on the two lines x = 0 and x = 1: the quadratic x (x - 1)
    vanishes on every node, so the m = 2 monomials are not unisolvent and P is
    rank-deficient.  The stencil takes m = 1 on the same nodes: its weights are
    the plain m = 1 solve, they reproduce every linear field exactly, and a
    generic stencil beside it keeps m = 2."""
    rng = np.random.default_rng(5)
    ys = np.sort(rng.uniform(-1.0, 1.0, 12))
    line = np.stack([np.r_[0.0, np.tile([0.0, 1.0], 6)[1:12]], np.r_[0.0, ys[1:]]])   # centre at the origin
    generic = rng.uniform(-1.0, 1.0, (2, 12)) + np.array([[3.0], [3.0]])
    generic[:, 0] = [3.0, 3.0]
    coords = np.concatenate([line, generic], 1)
    sten = np.array([np.arange(12), 12 + np.arange(12)])
    xi, _ = ow._scaled_offsets(coords, sten)
    assert list(ow.unisolvent(xi, 2)) == [False, True]
    W, m_used = ow.rbffd_weights_degree(coords, sten, 2)
    assert list(m_used) == [2 - 1, 2]
    W1 = ow.rbffd_weights(coords, sten[:1], 1)
    W2 = ow.rbffd_weights(coords, sten[1:], 2)
    for op in ("dx", "dy", "lap"):
        assert np.allclose(W[op][0], W1[op][0], rtol=0, atol=1e-12 * np.abs(W1[op][0]).max())
        assert np.allclose(W[op][1], W2[op][0], rtol=0, atol=1e-12 * np.abs(W2[op][0]).max())
    x, y = coords[:, sten[0]]
    for f, fx, fy in ((np.ones(12), 0.0, 0.0), (x, 1.0, 0.0), (y, 0.0, 1.0), (2 * x - 3 * y, 2.0, -3.0)):
        assert abs(W["dx"][0] @ f - fx) <= 1e-11 and abs(W["dy"][0] @ f - fy) <= 1e-11
        assert abs(W["lap"][0] @ f) <= 1e-10


def test_reduced_degree_agrees_with_the_singular_m3_systems_in_3d():
    """3D, m = 3 (n = 40): the stencils the oracle reduces to m = 2 are exactly
    those whose full m = 3 augmented system is singular to working precision
    (condition number above 1e14); every other stencil keeps m = 3 with a
    condition number far below that."""
    ns = nodesets.cube_spheres(n=14, n_holes=2, r_range=(0.1, 0.15), band=0.12, seed=nodesets.SEED_BASE + 21)
    st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, 40, normals=ns.normals)
    W = ow.all_weights(ns.coords, st, 3)
    xi, _ = ow._scaled_offsets(ns.coords, st["rbf_idx"])
    M, _ = ow.rbffd_system(xi, 3, ow.ops_for(3))
    cond = np.linalg.cond(M)
    reduced = W["rbf_m"] < 3
    assert reduced.any() and (~reduced).any()
    assert np.all(cond[reduced] > 1e14)
    assert np.all(cond[~reduced] < 1e10)
    assert np.all(W["rbf_m"][reduced] == 2)
    # the reduced stencils reproduce quadratics exactly
    x = ns.coords[:, st["rbf_idx"][reduced]]
    q = x[0] ** 2 + x[1] * x[2] - 2 * x[2] ** 2
    assert np.allclose((W["rbf"]["lap"][reduced] * q).sum(1), 2.0 - 4.0, atol=1e-7)
