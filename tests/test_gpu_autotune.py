"""Autotuned launch configurations against the FP64 oracle.

hsm_plan_autotune picks, per plan, the threads per kNN query, the lanes per
RBF-FD system (FP64 and FP32 + refinement), the arrangement of the FP64
weights (MON weights beside the kNN search plus one RBF-FD launch, one
grouped persistent launch for both groups, or both groups inside the stencil
build with the RBF-FD solve in 1, 2 or 4 chunks beside the kNN search) and
the apply block size.  Every
configuration it can pick must give the oracle's stencils (bit-exact), weights
(1e-10 FP64, 1e-5 FP32 + refinement) and operator values.  The tuner's own
choice is checked, then every variant is forced through its cache file."""
import os

import numpy as np
import pytest

from oracle import apply as oap
from oracle import stencils as ost
from oracle import weights as ow
from paper_2303_01760_gb300 import nodesets

from gpu_helpers import gpu_csr, to_dev

pytestmark = pytest.mark.gpu

BIT = {"dx": 1, "dy": 2, "dz": 4, "lap": 8}


def _check(plan, ns, st, W, prec, tol):
    import torch

    plan.build_stencils()
    assert plan.compute_weights(prec) == 0
    u, _ = nodesets.field_sincos(ns.coords)
    out = plan.apply(torch.from_numpy(u).cuda()).cpu().numpy()
    for k, op in enumerate(("dx", "dy", "lap")):
        rp, col, val = gpu_csr(plan, BIT[op])
        for grp, width in (("mon", 5), ("rbf", 12)):
            nodes = st[grp + "_nodes"]
            ix = rp[nodes][:, None] + np.arange(width)[None, :]
            assert np.array_equal(col[ix], st[grp + "_idx"])
            e = np.abs(val[ix] - W[grp][op]).max(1) / np.abs(W[grp][op]).max(1)
            assert e.max() <= tol, (grp, op, prec, e.max())
            ref = oap.apply_group(st[grp + "_idx"], W[grp][op], u)
            scale = (np.abs(W[grp][op]) * np.abs(u[st[grp + "_idx"]])).sum(1)
            assert np.all(np.abs(out[k, nodes] - ref) <= max(tol, 1e-12) * 10 * scale)


def test_autotuned_plan_and_every_variant_match_the_oracle(tmp_path):
    from paper_2303_01760_gb300 import hsm

    ns = nodesets.square_wall_band(n=60, seed=nodesets.SEED_BASE + 5)
    st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, 12, normals=ns.normals)
    W = ow.all_weights(ns.coords, st, 2)
    dv = to_dev(ns)

    def plan_with(cache):
        p = hsm.Plan(dv["coords"], dv["is_regular"], dv["is_boundary"], ns.h, m=2, normals=dv["normals"])
        p.build_stencils()
        p.autotune(cache)
        return p

    cache = str(tmp_path / "tune.txt")
    p = plan_with(cache)                      # times the variants, writes the cache
    _check(p, ns, st, W, hsm.HSM_PREC_FP64, 1e-10)
    _check(p, ns, st, W, hsm.HSM_PREC_FP32_REFINE, 1e-5)
    p.close()
    key, chosen = open(cache).read().split()
    assert len(chosen.split(",")) == 6
    # apply threads, FP64 lanes, kNN threads per query, FP32 lanes, weights
    # arrangement (0 split, 1 grouped launch, 2 in the build), chunks
    for t, l64, q, l32, ar, ch in ((64, 4, 2, 16, 1, 1), (128, 16, 4, 32, 0, 1), (256, 32, 1, 4, 1, 1),
                                   (256, 8, 1, 8, 0, 1), (128, 8, 4, 8, 1, 1), (128, 8, 2, 8, 2, 1),
                                   (256, 16, 1, 8, 2, 2), (64, 8, 4, 16, 2, 4)):
        with open(cache, "w") as f:
            f.write(f"{key} {t},{l64},{q},{l32},{ar},{ch}\n")
        p = plan_with(cache)                  # loads the forced variant
        _check(p, ns, st, W, hsm.HSM_PREC_FP64, 1e-10)
        _check(p, ns, st, W, hsm.HSM_PREC_FP32_REFINE, 1e-5)
        p.close()
    assert os.path.exists(cache)


@pytest.mark.parametrize("qt", [1, 2, 4])
@pytest.mark.parametrize("which", ["refined2d", "refined3d", "cube_m3"])
def test_knn_variants_match_the_oracle(which, qt):
    """Every kNN variant (1, 2 or 4 threads per query; a first window of rings
    0..R0 sized from the local spacing, then ring by ring) on h-refined sets,
    whose spacing varies by a factor of several inside one window and whose
    boundary stencils search from a point one local spacing inside, and on
    the 3D set with m = 3 (n = 40): every stencil equal to the oracle's, and
    the weights within 1e-10."""
    from paper_2303_01760_gb300 import hsm

    from test_gpu_weights import REFINED_2D, REFINED_3D

    if which == "refined2d":
        ns, m = nodesets.holes_refined(**REFINED_2D), 2
    elif which == "refined3d":
        ns, m = nodesets.holes_refined(**REFINED_3D), 2
    else:
        ns, m = nodesets.cube_spheres(n=14, n_holes=2, r_range=(0.1, 0.15), band=0.12,
                                      seed=nodesets.SEED_BASE + 21), 3
    n = ow.stencil_size(ns.dim, m)
    st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, n, normals=ns.normals,
                            spacing=ns.spacing)
    W = ow.all_weights(ns.coords, st, m)
    dv = to_dev(ns)
    p = hsm.Plan(dv["coords"], dv["is_regular"], dv["is_boundary"], ns.h, m=m, normals=dv["normals"],
                 spacing=dv["spacing"])
    p._dv = dv
    for bad in (0, 3, 32):
        with pytest.raises(hsm.HsmError):
            p.set_tuning(knn_qt=bad, rbf_lanes=8, rbf_lanes32=8, apply_threads=128, arrange=0)
    p.set_tuning(knn_qt=qt, rbf_lanes=8, rbf_lanes32=8, apply_threads=128, arrange=0)
    p.build_stencils()
    assert p.tuning()["knn_qt"] == qt
    assert p.compute_weights(hsm.HSM_PREC_FP64) == 0
    bits = {"dx": 1, "dy": 2, "dz": 4, "lap": 8}
    for op in ow.ops_for(ns.dim):
        rp, col, val = gpu_csr(p, bits[op])
        ix = rp[st["rbf_nodes"]][:, None] + np.arange(n)[None, :]
        assert np.array_equal(col[ix], st["rbf_idx"]), which
        e = np.abs(val[ix] - W["rbf"][op]).max(1) / np.abs(W["rbf"][op]).max(1)
        assert e.max() <= 1e-10, (which, op, e.max())
    p.close()


@pytest.mark.parametrize("chunks", [1, 2, 4])
@pytest.mark.parametrize("which", ["holes2d", "cube_m3"])
def test_weights_in_the_build_match_the_split_arrangement_and_the_oracle(which, chunks):
    """Arrangement 2: the stencil build solves the RBF-FD group in FP64 in
    `chunks` chunks, chunk c beside the kNN search of chunk c + 1, and the
    next FP64 weights call only reads the status words.  The weights must be
    bit-identical to the split arrangement's (the same solve, only its
    launches differ) and within 1e-10 of the oracle, on a 2D hybrid set and
    on the 3D m = 3 set (whose box-edge wall systems take the lower-degree
    retry after the in-build solve).  A second FP64 call, a call with
    node_status and an FP32 + refinement call solve again and agree."""
    import torch
    from paper_2303_01760_gb300 import hsm

    if which == "holes2d":
        ns, m = nodesets.square_holes(n=120, seed=nodesets.SEED_BASE + 9), 2
    else:
        ns, m = nodesets.cube_spheres(n=14, n_holes=2, r_range=(0.1, 0.15), band=0.12,
                                      seed=nodesets.SEED_BASE + 21), 3
    n = ow.stencil_size(ns.dim, m)
    st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, n, normals=ns.normals)
    W = ow.all_weights(ns.coords, st, m)
    dv = to_dev(ns)
    ops = ow.ops_for(ns.dim)
    bits = {"dx": 1, "dy": 2, "dz": 4, "lap": 8}

    def weights(arrange, ch):
        p = hsm.Plan(dv["coords"], dv["is_regular"], dv["is_boundary"], ns.h, m=m, normals=dv["normals"])
        p.set_tuning(knn_qt=2, rbf_lanes=8, rbf_lanes32=8, apply_threads=128, arrange=arrange, chunks=ch)
        p.build_stencils()
        code = p.compute_weights(hsm.HSM_PREC_FP64, allow_singular=True)
        out = {op: gpu_csr(p, bits[op]) for op in ops}
        return p, code, out, p.query()

    p0, c0, ref, q0 = weights(0, 1)
    p0.close()
    p2, c2, got, q2 = weights(2, chunks)
    assert (c2, q2) == (c0, q0)
    for op in ops:
        for a, b in zip(ref[op], got[op]):
            assert np.array_equal(a, b), (which, chunks, op)
        rp, col, val = got[op]
        ix = rp[st["rbf_nodes"]][:, None] + np.arange(n)[None, :]
        assert np.array_equal(col[ix], st["rbf_idx"])
        e = np.abs(val[ix] - W["rbf"][op]).max(1) / np.abs(W["rbf"][op]).max(1)
        assert e.max() <= 1e-10, (which, op, e.max())
    # a second FP64 call solves again (the build's status words are consumed)
    assert p2.compute_weights(hsm.HSM_PREC_FP64, allow_singular=True) == c0
    for op in ops:
        assert np.array_equal(gpu_csr(p2, bits[op])[2], ref[op][2])
    # per-node status needs the solve in the weights call
    p2.build_stencils()
    status = torch.full((ns.N,), 77, dtype=torch.uint8, device="cuda:0")
    assert p2.compute_weights(hsm.HSM_PREC_FP64, status, allow_singular=True) == c0
    assert int((status == 77).sum()) == 0
    for op in ops:
        assert np.array_equal(gpu_csr(p2, bits[op])[2], ref[op][2])
    # another precision after an in-build FP64 solve
    p2.build_stencils()
    assert p2.compute_weights(hsm.HSM_PREC_FP32_REFINE, allow_singular=True) == c0
    for op in ops:
        rp, col, val = gpu_csr(p2, bits[op])
        ix = rp[st["rbf_nodes"]][:, None] + np.arange(n)[None, :]
        e = np.abs(val[ix] - W["rbf"][op]).max(1) / np.abs(W["rbf"][op]).max(1)
        assert e.max() <= 1e-5, (which, op, e.max())
    p2.close()
