"""Failure paths of the CUDA library, each provoked without faulting the GPU:
a pressure solve capped below its tolerance, an FP32 factorisation that
cannot be refined, and a tensor-core pipeline whose loads are held back so
that its bounded waits run out."""
import time

import numpy as np
import pytest

from oracle import stencils as ost
from oracle import weights as ow
from paper_2303_01760_gb300 import nodesets

from gpu_helpers import gpu_csr, make_plan

pytestmark = pytest.mark.gpu


def test_krylov_cap_returns_notconv():
    """A pressure solve capped at 2 iterations with a tolerance of 1e-14 stops
    before converging: hsm_step reports HSM_ENOTCONV (5), and with the caller's
    consent the steps still run and leave finite fields."""
    import torch
    from paper_2303_01760_gb300 import hsm

    ns = nodesets.square_wall_band(n=20)
    plan, code, _ = make_plan(ns, m=2)
    assert code == 0
    dv = plan._dev
    st = hsm.Stepper(plan, 1e4, 0.71, 0.1 * ns.h ** 2 / 2, ns.T_ref, dv["bc"], dv["T_bc"], dv["normals"],
                     krylov_tol=1e-14, krylov_max_it=2)
    v = torch.zeros((2, ns.N), dtype=torch.float64, device="cuda:0")
    T = torch.where(dv["bc"] == 1, dv["T_bc"], torch.zeros_like(dv["T_bc"])).contiguous()
    p = torch.zeros(ns.N, dtype=torch.float64, device="cuda:0")
    with pytest.raises(hsm.HsmError) as e:
        st.step(v, T, p, 3)
    assert e.value.code == 5
    its, code = st.step(v, T, p, 3, allow_notconv=True)
    assert code == 5
    assert all(1 <= k <= 4 for k in its)
    assert bool(torch.isfinite(v).all() and torch.isfinite(T).all() and torch.isfinite(p).all())
    st.close()
    plan.close()


def test_fp32_refinement_falls_back_to_fp64():
    """Two scattered nodes 1e-4 h apart make the systems of the stencils that
    hold both ill-conditioned (kappa ~ 1e10, beyond FP32).  Most of them fail
    to refine and are re-solved in FP64 (status 2; on a GB300 8 of 10, the
    other two refined to convergence); all of them match the oracle to the
    accuracy kappa allows, and every other node is unaffected."""
    ns = nodesets.square_wall_band(n=20)
    sc = np.flatnonzero((ns.is_regular == 0) & (ns.is_boundary == 0))
    a, b = sc[0], sc[1]
    ns.coords[:, b] = ns.coords[:, a] + 1e-4 * ns.h * np.array([0.6, 0.8])
    plan, code, status = make_plan(ns, m=2, prec=1, node_status=True)
    assert code == 0
    status = status.cpu().numpy()
    st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, 12, normals=ns.normals)
    W = ow.all_weights(ns.coords, st, 2)
    both = np.any(st["rbf_idx"] == a, 1) & np.any(st["rbf_idx"] == b, 1)
    assert both.sum() >= 4
    sb = status[st["rbf_nodes"][both]]
    assert np.all(np.isin(sb, (0, 2)))
    assert np.sum(sb == 2) * 2 > len(sb)
    assert np.all(np.isin(status[st["rbf_nodes"][~both]], (0, 1)))
    rp, col, val = gpu_csr(plan, 8)
    ix = rp[st["rbf_nodes"]][:, None] + np.arange(12)[None, :]
    assert np.array_equal(col[ix], st["rbf_idx"])
    e = np.abs(val[ix] - W["rbf"]["lap"]).max(1) / np.abs(W["rbf"]["lap"]).max(1)
    assert e[both].max() <= 1e-3
    assert e[~both].max() <= 1e-5
    plan.close()


def test_mlp_forward_timeout_is_reported_and_recovers():
    """With its loads held back the fused tcgen05 forward pass never receives
    its inputs: the tensor-core and epilogue roles give up after their bounded
    waits, release the tensor memory and the call returns HSM_ETIMEOUT (6)
    within seconds.  The next call runs normally and gives the same outputs,
    bit for bit, as a call before the fault."""
    import torch
    from paper_2303_01760_gb300 import hsm

    mlp = hsm.MLP(24, 256, 3, 36, seed=11)
    X = torch.from_numpy(nodesets.seeded_uniform((300, 24), 5).astype(np.float32)).cuda()
    Y0 = mlp.predict(X).clone()
    mlp.inject_fault(hsm.HSM_FAULT_HOLD_MLP_LOADS)
    t0 = time.time()
    with pytest.raises(hsm.HsmError) as e:
        mlp.predict(X)
    assert e.value.code == 6
    assert time.time() - t0 < 60.0
    Y1 = mlp.predict(X)
    assert torch.equal(Y0, Y1)
    mlp.close()
