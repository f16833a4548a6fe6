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
