"""The allocation-free weight entry point against the allocating plan path.

Some callers cannot allocate device memory while they run: an application
that hands all device memory to its own pool at start-up, or a real-time loop
in which an allocation could stall or fail.  hsm_rbf_weights_fp32r_noalloc
serves them: the caller passes stencils, coordinates and output buffers, and
the library's scratch is a fixed static device array.  This file runs last so
that a failure here leaves every other test already run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_FP32R = 1e-5  # relative weight error per stencil, as for the FP32-refinement path


def _plan_rbf_rows(ns):
    from gpu_helpers import make_plan
    from paper_2303_01760_gb300 import hsm

    plan, code, _ = make_plan(ns, m=2, prec=hsm.HSM_PREC_FP32_REFINE)
    assert code == 0
    idx, w = None, []
    for op in (hsm.HSM_DX, hsm.HSM_DY, hsm.HSM_LAP):
        rp, col, val = [t.cpu().numpy() for t in plan.export_csr(op)]
        widths = np.diff(rp)
        rows = np.flatnonzero(widths == 12)
        ix = rp[rows][:, None] + np.arange(12)[None, :]
        idx = col[ix]
        w.append(val[ix])
    plan.close()
    return idx, np.stack(w)  # [count, 12], [3, count, 12]


def test_noalloc_weights_match_plan_path_on_two_calls():
    import torch
    from paper_2303_01760_gb300 import hsm, nodesets

    ns = nodesets.square_wall_band(n=40)
    idx, w_plan = _plan_rbf_rows(ns)
    count = idx.shape[0]
    coords = torch.from_numpy(ns.coords).cuda()
    sten = torch.from_numpy(np.ascontiguousarray(idx.T.astype(np.int32))).cuda()   # [n, count]
    status = torch.full((ns.N,), 77, dtype=torch.uint8, device="cuda:0")
    mask = hsm.HSM_DX | hsm.HSM_DY | hsm.HSM_LAP
    for call in range(2):
        w = torch.full((3, 12, count), np.nan, dtype=torch.float64, device="cuda:0")
        code = hsm.rbf_weights_fp32r_noalloc(2, 2, 12, mask, coords, sten, w, status)
        torch.cuda.synchronize()
        assert code == 0, hsm.last_error()
        got = w.cpu().numpy().transpose(0, 2, 1)                     # [3, count, 12]
        rel = np.abs(got - w_plan).max(2) / np.abs(w_plan).max(2)
        assert rel.max() <= TOL_FP32R, (call, rel.max())
        st = status.cpu().numpy()
        assert np.all(np.isin(st, (0, 2)))
        assert np.all(st[idx[:, 0]] != 255)


def test_noalloc_allocates_nothing_and_resolves_ill_conditioned_systems_in_fp64():
    """Two scattered nodes 1e-4 h apart make the systems that hold both too
    ill-conditioned for FP32 refinement: some must come back re-solved in
    FP64 (status 2), and every system must match the oracle's weights (to
    1e-3 where kappa ~ 1e10 allows no better, 1e-5 elsewhere).  A warm call
    leaves the device's free memory unchanged."""
    import torch
    from oracle import stencils as ost
    from oracle import weights as ow
    from paper_2303_01760_gb300 import hsm, nodesets

    ns = nodesets.square_wall_band(n=20)
    sc = np.flatnonzero((ns.is_regular == 0) & (ns.is_boundary == 0))
    a, b = sc[0], sc[1]
    ns.coords[:, b] = ns.coords[:, a] + 1e-4 * ns.h * np.array([0.6, 0.8])
    st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, 12, normals=ns.normals)
    W = ow.all_weights(ns.coords, st, 2)
    idx = st["rbf_idx"]                                   # [count, 12], row-major per stencil
    count = idx.shape[0]
    coords = torch.from_numpy(np.ascontiguousarray(ns.coords)).cuda()
    sten = torch.from_numpy(np.ascontiguousarray(idx.T.astype(np.int32))).cuda()
    status = torch.full((ns.N,), 77, dtype=torch.uint8, device="cuda:0")
    w = torch.full((3, 12, count), np.nan, dtype=torch.float64, device="cuda:0")
    mask = hsm.HSM_DX | hsm.HSM_DY | hsm.HSM_LAP
    assert hsm.rbf_weights_fp32r_noalloc(2, 2, 12, mask, coords, sten, w, status) == 0, hsm.last_error()
    torch.cuda.synchronize()
    w.fill_(np.nan)
    status.fill_(77)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    code = hsm.rbf_weights_fp32r_noalloc(2, 2, 12, mask, coords, sten, w, status)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert code == 0, hsm.last_error()
    assert free1 == free0, (free0, free1)
    s = status.cpu().numpy()
    both = np.any(idx == a, 1) & np.any(idx == b, 1)
    assert both.sum() >= 4
    assert np.sum(s[st["rbf_nodes"][both]] == 2) >= 1     # the FP64 re-solve ran
    assert np.all(np.isin(s[st["rbf_nodes"]], (0, 2)))
    got = w.cpu().numpy().transpose(0, 2, 1)              # [3, count, 12]
    for k, op in enumerate(("dx", "dy", "lap")):
        ref = W["rbf"][op]
        e = np.abs(got[k] - ref).max(1) / np.abs(ref).max(1)
        assert e[both].max() <= 1e-3, (op, e[both].max())
        assert e[~both].max() <= TOL_FP32R, (op, e[~both].max())


def test_noalloc_rejects_sizes_without_an_fp64_shape_and_bad_ids():
    """A 2D m=1 stencil of 100 nodes fits the FP32 pass but not the FP64
    re-solve: rejected with HSM_EINVAL before any work.  A stencil id outside
    [0, n_nodes) is rejected with HSM_EBOUNDS before any weight kernel runs;
    the outputs are left as they were."""
    import torch
    from paper_2303_01760_gb300 import hsm

    N = 256
    coords = torch.rand((2, N), dtype=torch.float64, device="cuda:0")
    sten = torch.arange(100, dtype=torch.int32, device="cuda:0").reshape(100, 1).contiguous()
    w = torch.zeros((3, 100, 1), dtype=torch.float64, device="cuda:0")
    code = hsm.rbf_weights_fp32r_noalloc(2, 1, 100, 11, coords, sten, w, None)
    assert code == 1
    assert "FP64" in hsm.last_error()

    sten = torch.arange(24, dtype=torch.int32, device="cuda:0").reshape(12, 2).contiguous()
    sten[5, 1] = N                                         # one past the end
    w = torch.full((3, 12, 2), np.nan, dtype=torch.float64, device="cuda:0")
    status = torch.full((N,), 77, dtype=torch.uint8, device="cuda:0")
    code = hsm.rbf_weights_fp32r_noalloc(2, 2, 12, 11, coords, sten, w, status)
    torch.cuda.synchronize()
    assert code == hsm.HSM_EBOUNDS, hsm.last_error()
    assert bool(torch.isnan(w).all())
    assert bool((status == 77).all())
    sten[5, 1] = -1
    assert hsm.rbf_weights_fp32r_noalloc(2, 2, 12, 11, coords, sten, w, status) == hsm.HSM_EBOUNDS


def test_noalloc_rejects_batches_beyond_its_scratch():
    import torch
    from paper_2303_01760_gb300 import hsm

    coords = torch.zeros((2, 16), dtype=torch.float64, device="cuda:0")
    sten = torch.zeros((12, 1), dtype=torch.int32, device="cuda:0")
    w = torch.zeros((3, 12, 1), dtype=torch.float64, device="cuda:0")
    code = hsm.lib.hsm_rbf_weights_fp32r_noalloc(2, 2, 12, 11, hsm.ptr(coords), 16, hsm.ptr(sten),
                                                 hsm.HSM_NOALLOC_MAX_SYSTEMS + 1, hsm.ptr(w), None,
                                                 hsm.stream_handle())
    assert code == 1
    assert "HSM_NOALLOC_MAX_SYSTEMS" in hsm.last_error()
