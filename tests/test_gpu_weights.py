"""CUDA path vs the FP64 oracle: stencils, weights and operator application
(Eq. 1, Section 2 and 2.1), called through the C ABI."""
import numpy as np
import pytest

from oracle import apply as oap
from oracle import stencils as ost
from oracle import weights as ow
from paper_2303_01760_gb300 import nodesets

from gpu_helpers import gpu_csr, make_plan

pytestmark = pytest.mark.gpu

BIT = {"dx": 1, "dy": 2, "dz": 4, "lap": 8}
TOL_FP64 = 1e-10      # relative weight error per stencil and operator, FP64 path
TOL_FP32R = 1e-5      # FP32 factorisation + FP64 refinement


def _rows(rp, col, val, nodes, width):
    ix = rp[nodes][:, None] + np.arange(width)[None, :]
    return col[ix], val[ix]


def _rel(a, b):
    return np.abs(a - b).max(1) / np.abs(b).max(1)


def _oracle_cond(ns, st, m):
    xi, _ = ow._scaled_offsets(ns.coords, st["rbf_idx"])
    M, _ = ow.rbffd_system(xi, m, ow.ops_for(ns.dim))
    return np.linalg.cond(M)


def _check_plan(ns, m, prec=0, centers=None, tol=TOL_FP64, apply_check=True, singular_ok=False):
    import torch

    dim = ns.dim
    n = ow.stencil_size(dim, m)
    ops = ow.ops_for(dim)
    plan, code, status = make_plan(ns, m=m, prec=prec, node_status=True)
    st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, n, centers=centers,
                            normals=ns.normals, spacing=ns.spacing)
    if singular_ok:
        # nodes whose system is singular to working precision must be flagged
        # (status 255, zero weights); well-conditioned ones must not be
        cond = _oracle_cond(ns, st, m)
        flagged = status.cpu().numpy()[st["rbf_nodes"]] == 255
        assert np.all(flagged[cond > 1e14])
        assert np.all(cond[flagged] > 1e8)
        assert code == (4 if flagged.any() else 0)
        keep = ~flagged
        st = dict(st, rbf_nodes=st["rbf_nodes"][keep], rbf_idx=st["rbf_idx"][keep])
        st["demoted"] = np.intersect1d(st["demoted"], np.r_[st["mon_nodes"], st["rbf_nodes"]])
        centers = np.r_[st["mon_nodes"], st["rbf_nodes"]] if flagged.any() else centers
    else:
        assert code == 0
    W = ow.all_weights(ns.coords, st, m)
    q = plan.query()
    if centers is None and not singular_ok:
        assert q["n_mon"] == len(st["mon_nodes"])
        assert q["n_demoted"] == len(st["demoted"])
    status = status.cpu().numpy()
    # stencils on which the degree-m monomials are not unisolvent take a lower
    # degree on the same nodes (oracle and GPU alike), status 4
    reduced = st["rbf_nodes"][W["rbf_m"] < m] if "rbf_m" in W else np.zeros(0, dtype=np.int64)
    assert np.all(status[reduced] == 4)
    assert not np.any(status[np.setdiff1d(st["rbf_nodes"], reduced)] == 4)
    if prec == 0:
        assert np.all(status[st["mon_nodes"]] == 0)
        assert np.all(status[np.setdiff1d(st["demoted"], reduced)] == 1)
    else:
        assert np.all(np.isin(status[st["rbf_nodes"]], (0, 1, 2, 4)))
    worst = {}
    for op in ops:
        rp, col, val = gpu_csr(plan, BIT[op])
        for grp, width in (("mon", 2 * dim + 1), ("rbf", n)):
            nodes = st[grp + "_nodes"]
            if len(nodes) == 0:
                continue
            c, v = _rows(rp, col, val, nodes, width)
            assert np.array_equal(rp[nodes + 1] - rp[nodes], np.full(len(nodes), width))
            assert np.array_equal(c, st[grp + "_idx"]), f"{grp} stencil mismatch"
            e = _rel(v, W[grp][op])
            worst[(grp, op)] = float(e.max())
            assert e.max() <= tol, (grp, op, e.max(), int(np.argmax(e)))
    if apply_check:
        u, _ = nodesets.field_sincos(ns.coords) if dim == 2 else nodesets.field_random_smooth(ns.coords)
        ut = torch.from_numpy(u).cuda()
        out = plan.apply(ut).cpu().numpy()
        out32 = plan.apply(ut.float()).cpu().numpy()
        for k, op in enumerate(ops):
            for grp in ("mon", "rbf"):
                nodes = st[grp + "_nodes"]
                if len(nodes) == 0:
                    continue
                ref = oap.apply_group(st[grp + "_idx"], W[grp][op], u)
                scale = (np.abs(W[grp][op]) * np.abs(u[st[grp + "_idx"]])).sum(1)
                assert np.all(np.abs(out[k, nodes] - ref) <= max(tol, 1e-12) * 10 * scale)
                # FP32 inputs, weights and sums: (W + 2) unit roundoffs of sum |w u|
                width = st[grp + "_idx"].shape[1]
                assert np.all(np.abs(out32[k, nodes] - ref) <= ((width + 2) * 2.0 ** -24 + 2 * tol) * scale)
    plan.close()
    return worst


def test_square_wall_band_fp64_full():
    """Unit square, lattice h=1/40 inside, Poisson-disk band along the walls,
    m=2, n=12: every stencil and weight against the oracle."""
    _check_plan(nodesets.square_wall_band(n=40), m=2)


def test_square_wall_band_m4():
    _check_plan(nodesets.square_wall_band(n=30, seed=nodesets.SEED_BASE + 11), m=4)


def test_all_regular_and_all_scattered():
    ns = nodesets.square_wall_band(n=32, wall_band=0.0)
    _check_plan(ns, m=2)
    _check_plan(ns.all_scattered(), m=2)


def test_cube_spheres_small_m2_m3():
    """3D: unit cube minus 2 spheres, m=2 (n=20) and m=3 (n=40).  With m=3 the
    wall nodes next to a box edge have one-sided stencils that span only three
    lattice layers across the edge, so the cubic monomials are not unisolvent
    there; those nodes take m = 2 on the same 40 nodes (status 4), and every
    node, those included, matches the oracle's weights."""
    ns = nodesets.cube_spheres(n=14, n_holes=2, r_range=(0.1, 0.15), band=0.12, seed=nodesets.SEED_BASE + 21)
    _check_plan(ns, m=2)
    _check_plan(ns, m=3)


def test_fp32_refinement_within_tolerance():
    ns = nodesets.square_wall_band(n=40)
    w = _check_plan(ns, m=2, prec=1, tol=TOL_FP32R)
    assert max(w.values()) <= TOL_FP32R


def test_fp32_refinement_m4_and_3d():
    _check_plan(nodesets.square_wall_band(n=30, seed=nodesets.SEED_BASE + 11), m=4, prec=1, tol=TOL_FP32R)
    ns = nodesets.cube_spheres(n=14, n_holes=2, r_range=(0.1, 0.15), band=0.12, seed=nodesets.SEED_BASE + 21)
    _check_plan(ns, m=3, prec=1, tol=TOL_FP32R)


def test_irregular_250k_sampled():
    """The 2D irregular workload at full size (unit square minus 8 holes,
    h=0.002): sampled nodes compared one by one with the oracle."""
    ns = nodesets.cached(nodesets.square_holes)
    rng = np.random.default_rng(123)
    centers = np.unique(np.r_[rng.choice(ns.N, 3000, replace=False), np.flatnonzero(ns.is_boundary)[:500]])
    _check_plan(ns, m=2, centers=centers)


@pytest.mark.parametrize("m,all_rbffd", [(4, False), (2, True)])
def test_irregular_250k_sampled_m4_and_all_rbffd(m, all_rbffd):
    """The same full-size set with m = 4 (n = 30), and with every node forced
    to RBF-FD (the 100 % end of the scattered-fraction sweep): sampled nodes
    against the oracle."""
    ns = nodesets.cached(nodesets.square_holes)
    if all_rbffd:
        ns = ns.all_scattered()
    rng = np.random.default_rng(124)
    centers = np.unique(np.r_[rng.choice(ns.N, 2000, replace=False), np.flatnonzero(ns.is_boundary)[:300]])
    _check_plan(ns, m=m, centers=centers)


def test_tiled_7m_sampled():
    """The 8M-node 2D shape, 30 % scattered: 12 x 12 tiled copies of a unit
    square minus 8 holes (lattice h = 1/250, band 0.09), 7,339,248 nodes, the
    plan the benchmark times for its apply roofline.  Sampled nodes against
    the oracle, FP64 and FP32 + refinement weights and the f64/f32 apply."""
    base = nodesets.cached(nodesets.square_holes, n=250, band=0.09)
    ns = nodesets.tiled(base, 12, 12)
    assert ns.N == 7339248
    rng = np.random.default_rng(125)
    bnd = np.flatnonzero(ns.is_boundary)
    centers = np.unique(np.r_[rng.choice(ns.N, 2500, replace=False), rng.choice(bnd, 500, replace=False)])
    _check_plan(ns, m=2, centers=centers)
    _check_plan(ns, m=2, prec=1, tol=TOL_FP32R, centers=centers, apply_check=False)


def test_duplicate_nodes_are_reported_singular():
    """Two scattered nodes at the same position make their RBF-FD systems
    singular: the call reports HSM_ESINGULAR and marks those nodes 255
    without faulting."""
    ns = nodesets.square_wall_band(n=20)
    sc = np.flatnonzero((ns.is_regular == 0) & (ns.is_boundary == 0))
    ns.coords[:, sc[1]] = ns.coords[:, sc[0]]
    plan, code, status = make_plan(ns, m=2, node_status=True)
    assert code == 4
    status = status.cpu().numpy()
    assert status[sc[0]] == 255 and status[sc[1]] == 255
    assert np.sum(status == 255) < ns.N // 4
    plan.close()


def test_invalid_arguments_rejected_before_launch():
    import torch
    from paper_2303_01760_gb300 import hsm

    ns = nodesets.square_wall_band(n=10)
    c = torch.from_numpy(ns.coords).cuda()
    r = torch.from_numpy(ns.is_regular).cuda()
    with pytest.raises(hsm.HsmError) as e:
        hsm.Plan(c, r, None, ns.h, m=2, n=3)
    assert e.value.code == 1
    with pytest.raises(hsm.HsmError):
        hsm.Plan(c, r, None, ns.h, m=2, op_mask=hsm.HSM_DZ)
    p = hsm.Plan(c, r, None, ns.h, m=2)
    with pytest.raises(hsm.HsmError) as e:
        p.compute_weights()
    assert e.value.code == 8
    p.close()


def test_mon_weights_on_slightly_perturbed_lattice():
    """Regular nodes within the lattice tolerance but off exact alignment take
    the general MON elimination instead of the per-axis closed form; both must
    match the oracle's solve of the same system."""
    ns = nodesets.square_wall_band(n=24, wall_band=0.0)
    rng = np.random.default_rng(8)
    ns.coords = ns.coords + rng.uniform(-1e-9, 1e-9, ns.coords.shape) * ns.h
    _check_plan(ns, m=2)


def test_mon_weights_of_the_grouped_launch_match_the_oracle():
    """The MON weights come from the grouped weights launch (MON chunks and
    RBF-FD batches drawn from one work queue), with and without a node-status
    request; they match the oracle, and the two calls agree bit for bit, on
    exact, perturbed and banded lattices."""
    base = nodesets.square_wall_band(n=24, wall_band=0.0)
    pert = nodesets.square_wall_band(n=24, wall_band=0.0)
    rng = np.random.default_rng(9)
    pert.coords = pert.coords + rng.uniform(-1e-9, 1e-9, pert.coords.shape) * pert.h
    for ns in (nodesets.square_wall_band(n=40), base, pert):
        plan_a, code_a, _ = make_plan(ns, m=2)
        plan_b, code_b, _ = make_plan(ns, m=2, node_status=True)
        assert code_a == code_b == 0
        st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, 12, normals=ns.normals)
        W = ow.all_weights(ns.coords, st, 2)
        nodes = st["mon_nodes"]
        assert len(nodes) > 0
        for op in ow.ops_for(2):
            rp, col, val = gpu_csr(plan_a, BIT[op])
            _, _, val_b = gpu_csr(plan_b, BIT[op])
            assert np.array_equal(val, val_b)
            c, v = _rows(rp, col, val, nodes, 5)
            assert np.array_equal(c, st["mon_idx"])
            assert _rel(v, W["mon"][op]).max() <= TOL_FP64
        plan_a.close()
        plan_b.close()


def test_sparse_lattice_takes_the_hashed_map():
    """Two copies of a wall-band set 400 lattice spacings apart: the lattice's
    extents hold far more than 4N + 1024 points, so the build keeps its map
    in the hash instead of the dense array.  Stencils and weights must still
    match the oracle."""
    import dataclasses

    a = nodesets.square_wall_band(n=40)
    shift = 400 * a.h
    ns = dataclasses.replace(
        a, name="two copies",
        coords=np.concatenate([a.coords, a.coords + shift], axis=1),
        is_regular=np.concatenate([a.is_regular, a.is_regular]),
        is_boundary=np.concatenate([a.is_boundary, a.is_boundary]),
        normals=np.concatenate([a.normals, a.normals], axis=1),
        bc=np.concatenate([a.bc, a.bc]), T_bc=np.concatenate([a.T_bc, a.T_bc]))
    lattice_points = (401 + 40) ** 2
    assert lattice_points > 4 * ns.N + 1024
    _check_plan(ns, m=2)


REFINED_2D = dict(n=40, n_holes=2, r_range=(0.1, 0.15), delta_h=4.0, seed=nodesets.SEED_BASE + 60)
REFINED_3D = dict(dim=3, n=12, n_holes=1, r_range=(0.15, 0.2), delta_h=3.0, ratio=2.0, seed=nodesets.SEED_BASE + 61)


def test_refined_sets_2d_and_3d():
    """h-refined sets (Sections 4.2 and 4.3: spacing h_r/3 in 2D and h_r/2 in
    3D at the holes), boundary stencils searched one local spacing inside:
    every stencil and weight against the oracle, in FP64 and FP32 + refinement
    (the coarse 3D set included: with the spacing-aware fill every one of its
    m = 2 systems is regular, the largest condition number about 4.4e3)."""
    ns2 = nodesets.holes_refined(**REFINED_2D)
    _check_plan(ns2, m=2)
    _check_plan(ns2, m=2, prec=1, tol=TOL_FP32R)
    _check_plan(ns2.all_scattered(), m=2)
    _check_plan(nodesets.holes_refined(**REFINED_3D), m=2)


def test_setting_the_spacing_rebuilds_the_boundary_stencils():
    """A plan built with h_regular, then given the local spacing: the next
    build (a fresh capture of the build graph) takes the new search points,
    and clearing the spacing brings the old stencils back."""
    import torch
    from paper_2303_01760_gb300 import hsm

    ns = nodesets.holes_refined(**REFINED_2D)
    d = {k: torch.from_numpy(np.ascontiguousarray(getattr(ns, k))).cuda()
         for k in ("coords", "is_regular", "is_boundary", "normals", "spacing")}
    plan = hsm.Plan(d["coords"], d["is_regular"], d["is_boundary"], ns.h, m=2, normals=d["normals"])
    bnd = np.flatnonzero(ns.is_boundary)
    want = {}
    for key, sp in (("lattice", None), ("local", ns.spacing)):
        st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, 12, centers=bnd,
                                normals=ns.normals, spacing=sp)
        want[key] = st["rbf_idx"]
    assert not np.array_equal(want["lattice"], want["local"])
    for key, sp in (("lattice", None), ("local", d["spacing"]), ("lattice", None)):
        plan.set_spacing(sp)
        plan.build_stencils()
        plan.compute_weights(hsm.HSM_PREC_FP64)
        rp, col, val = gpu_csr(plan, BIT["dx"])
        c, _ = _rows(rp, col, val, bnd, 12)
        assert np.array_equal(c, want[key]), key
    plan.close()
