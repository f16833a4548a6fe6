"""Learned weights (the specification's predictor; no counterpart in the
paper): tensor-core MLP gradients and forward pass against the FP64 oracle,
the FP64 consistency projection against the oracle's, and the trained
predictor end to end (exact monomial reproduction, fallback, accuracy)."""
import numpy as np
import pytest

from oracle import learned as ol
from oracle import stencils as ost
from oracle import weights as ow
from paper_2303_01760_gb300 import nodesets

from gpu_helpers import make_plan

pytestmark = pytest.mark.gpu

H, L = 256, 3
TOL_BF16_GRAD = 5e-2   # BF16 operands/activations, FP32 accumulation, 4 layers
TOL_BF16_FWD = 2e-2


def _dataset(seeds, n=60, jitters=(0.0, 0.1, 0.2, 0.3)):
    """Features/labels of interior stencils of Poisson-disk sets, from the
    library's own FP64 weights (the plain solver)."""
    import torch

    Xs, Ys = [], []
    for sd in seeds:
        for j in jitters:
            ns = nodesets.square_all_scattered(n=n, seed=sd, jitter=j)
            plan, code, _ = make_plan(ns, m=2)
            assert code == 0
            X, Y = plan.learned_data()
            Xs.append(X)
            Ys.append(Y)
            plan.close()
    return torch.cat(Xs), torch.cat(Ys)


def _oracle_params(mlp):
    from paper_2303_01760_gb300 import hsm

    return hsm.unpack_params(mlp.get_params(), 24, H, L, 36)


def test_mlp_gradients_and_forward_match_oracle():
    from paper_2303_01760_gb300 import hsm

    X, Y = _dataset([nodesets.SEED_BASE + 60], jitters=(0.2,))
    X, Y = X[:300].contiguous(), Y[:300].contiguous()
    mlp = hsm.MLP(24, H, L, 36, seed=3)
    P = _oracle_params(mlp)
    Xn, Yn = X.double().cpu().numpy(), Y.double().cpu().numpy()
    loss_ref, g_ref = ol.loss_and_grad(P, Xn, Yn)
    loss, g = mlp.grad(X, Y)
    assert abs(loss - loss_ref) <= TOL_BF16_FWD * loss_ref
    G = hsm.unpack_params(g, 24, H, L, 36)
    for (gw, gb), (rw, rb) in zip(G, g_ref):
        ew = np.linalg.norm(gw - rw) / np.linalg.norm(rw)
        eb = np.linalg.norm(gb - rb) / np.linalg.norm(rb)
        assert ew <= TOL_BF16_GRAD and eb <= TOL_BF16_GRAD, (ew, eb)
    out_ref, _, _ = ol.forward(P, Xn)
    out = mlp.predict(X).double().cpu().numpy()
    assert np.abs(out - out_ref).max() <= TOL_BF16_FWD * np.abs(out_ref).max()
    mlp.close()


def test_learned_weights_end_to_end():
    import torch
    from paper_2303_01760_gb300 import hsm

    Xtr, Ytr = _dataset([nodesets.SEED_BASE + 61, nodesets.SEED_BASE + 62])
    mlp = hsm.MLP(24, H, L, 36, seed=5)
    log = mlp.train(Xtr, Ytr, steps=1500, batch=1024, lr=1e-3, seed=11)
    assert log[-50:].mean() < 0.05 * log[:10].mean()

    ns = nodesets.square_all_scattered(n=50, seed=nodesets.SEED_BASE + 63, jitter=0.15)
    plan, code, status = make_plan(ns, m=2, prec=0)
    plan.attach(mlp)
    # the projection path itself: no batch validation here
    plan.set_learned_gate(samples=0)
    st = torch.full((ns.N,), 77, dtype=torch.uint8, device="cuda:0")
    code = plan.compute_weights(hsm.HSM_PREC_LEARNED, st)
    assert code == 0
    assert plan.learned_gate()[:2] == (-1.0, False)
    q = plan.query()
    status = st.cpu().numpy()
    # oracle: stencils, exact weights, and the projection of the GPU's own MLP output
    stn = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, 12, normals=ns.normals)
    inner = ns.is_boundary[stn["rbf_nodes"]] == 0
    nodes, idx = stn["rbf_nodes"][inner], stn["rbf_idx"][inner]
    W = ow.rbffd_weights(ns.coords, idx, 2)
    Xte, _ = plan.learned_data(labels=False)
    Ypred = mlp.predict(Xte).double().cpu().numpy()
    w_proj, accept = ol.learned_weights(ns.coords, idx, 2, Ypred)
    # GPU weights
    got = {}
    for op, bit in (("dx", 1), ("dy", 2), ("lap", 8)):
        rp, col, val = [t.cpu().numpy() for t in plan.export_csr(bit)]
        ix = rp[nodes][:, None] + np.arange(12)[None, :]
        assert np.array_equal(col[ix], idx)
        got[op] = val[ix]
    gpu_accept = status[nodes] == hsm.HSM_NODE_OK
    fallback = status[nodes] == hsm.HSM_NODE_LEARNED_SOLVE
    assert np.all(gpu_accept | fallback)
    # the fallback decision matches the oracle's (same predictions, same rule)
    assert np.mean(gpu_accept == accept) > 0.995
    both = gpu_accept & accept
    for op in ("dx", "dy", "lap"):
        scale = np.abs(w_proj[op][both]).max(1)
        # projection parity: FP64 on both sides from the same predictions
        assert (np.abs(got[op][both] - w_proj[op][both]).max(1) / scale).max() <= 1e-10
        # fallback nodes carry the direct-solve weights
        if fallback.any():
            e = np.abs(got[op][fallback] - W[op][fallback]).max(1) / np.abs(W[op][fallback]).max(1)
            assert e.max() <= 1e-10
    # every accepted stencil reproduces all monomials of degree <= 2 exactly
    xi, s = ow._scaled_offsets(ns.coords, idx[both])
    Pm, lp = ol.constraint_system(xi, 2, ("dx", "dy", "lap"))
    wsc = np.stack([got["dx"][both] * s[:, None], got["dy"][both] * s[:, None], got["lap"][both] * s[:, None] ** 2], 2)
    assert ol.post_residual(wsc, Pm, lp).max() <= 1e-9
    assert q["n_fallback"] == int(np.sum(status == hsm.HSM_NODE_LEARNED_SOLVE))
    # accuracy on u = sin(pi x) cos(pi y): learned + projected against the direct solve
    u, der = nodesets.field_sincos(ns.coords)
    err_l = np.abs((got["lap"] * u[idx]).sum(1) - der["lap"][nodes])
    err_d = np.abs((W["lap"] * u[idx]).sum(1) - der["lap"][nodes])
    deep = np.minimum(ns.coords[:, nodes], 1 - ns.coords[:, nodes]).min(0) > 0.15
    rel_w = np.median(np.abs(got["lap"][both] - W["lap"][both]).max(1) / np.abs(W["lap"][both]).max(1))
    print(f"accept {gpu_accept.mean():.3f}  median rel weight diff {rel_w:.2e}  "
          f"lap err learned {err_l[deep].max():.3e} direct {err_d[deep].max():.3e}")
    assert gpu_accept.mean() > 0.5
    assert err_l[deep].max() <= 5.0 * err_d[deep].max()
    plan.close()
    mlp.close()


def test_learned_batch_gate():
    """Batch validation of the learned weights: S stencils spread evenly over
    the interior (learned) positions are solved directly; the mean over the
    accepted ones of max|w_learned - w_direct| / max|w_direct| is the batch
    error.  It matches the oracle's value for the same samples and
    predictions; above the tolerance the whole batch takes the direct solve."""
    import torch
    from paper_2303_01760_gb300 import hsm

    Xtr, Ytr = _dataset([nodesets.SEED_BASE + 61])
    mlp = hsm.MLP(24, H, L, 36, seed=5)
    mlp.train(Xtr, Ytr, steps=300, batch=1024, lr=1e-3, seed=11)
    ns = nodesets.square_all_scattered(n=50, seed=nodesets.SEED_BASE + 63, jitter=0.15)
    stn = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, 12, normals=ns.normals)
    inner = ns.is_boundary[stn["rbf_nodes"]] == 0
    learn_pos = np.flatnonzero(inner)          # interior positions of the RBF-FD group, ascending
    W_all = ow.rbffd_weights(ns.coords, stn["rbf_idx"], 2)
    S = 64
    samp = learn_pos[(np.arange(S) * len(learn_pos)) // S]

    # a loose tolerance: the batch passes; the samples carry the direct weights
    plan, _, _ = make_plan(ns, m=2, prec=0)
    plan.attach(mlp)
    plan.set_learned_gate(tol=10.0, samples=S)
    st = torch.full((ns.N,), 77, dtype=torch.uint8, device="cuda:0")
    assert plan.compute_weights(hsm.HSM_PREC_LEARNED, st) == 0
    err, failed, n_acc = plan.learned_gate()
    assert not failed
    Xte, _ = plan.learned_data(labels=False)
    Ypred = mlp.predict(Xte).double().cpu().numpy()
    w_proj, accept = ol.learned_weights(ns.coords, stn["rbf_idx"][inner], 2, Ypred)
    k = np.searchsorted(learn_pos, samp)       # the samples' rows among the learned stencils
    ok = accept[k]
    rel = np.stack([np.abs(w_proj[op][k] - W_all[op][samp]).max(1) for op in ("dx", "dy", "lap")]).max(0)
    den = np.stack([np.abs(W_all[op][samp]).max(1) for op in ("dx", "dy", "lap")]).max(0)
    ref_err = float(np.mean((rel / den)[ok]))
    if n_acc == int(ok.sum()):
        # the same samples on both sides (the acceptance rule agrees)
        assert abs(err - ref_err) <= 1e-7 * ref_err
    else:
        assert abs(n_acc - int(ok.sum())) <= 2 and abs(err / ref_err - 1.0) <= 0.2
    status = st.cpu().numpy()
    nodes = stn["rbf_nodes"]
    assert np.all(status[nodes[samp[ok]]] == hsm.HSM_NODE_LEARNED_SOLVE)
    assert plan.query()["n_fallback"] == int(np.sum(status == hsm.HSM_NODE_LEARNED_SOLVE))
    plan.close()

    # the default tolerance (1e-3): this briefly trained predictor fails it,
    # and every RBF-FD stencil carries the direct-solve weights
    plan, _, _ = make_plan(ns, m=2, prec=0)
    plan.attach(mlp)
    plan.set_learned_gate(samples=S)
    st = torch.full((ns.N,), 77, dtype=torch.uint8, device="cuda:0")
    assert plan.compute_weights(hsm.HSM_PREC_LEARNED, st) == 0
    err2, failed2, _ = plan.learned_gate()
    assert failed2 and err2 == err and err2 > 1e-3
    status = st.cpu().numpy()
    assert np.all(status[nodes] == hsm.HSM_NODE_LEARNED_SOLVE)
    assert plan.query()["n_fallback"] == len(nodes)
    for op, bit in (("dx", 1), ("dy", 2), ("lap", 8)):
        rp, col, val = [t.cpu().numpy() for t in plan.export_csr(bit)]
        ix = rp[nodes][:, None] + np.arange(12)[None, :]
        e = np.abs(val[ix] - W_all[op]).max(1) / np.abs(W_all[op]).max(1)
        assert e.max() <= 1e-10
    plan.close()
    mlp.close()


def test_fused_forward_spans_many_tiles():
    """The fused tcgen05 forward pass over 1,000 128-row tiles plus a ragged
    tail (rows % 128 = 37), against the FP64 oracle forward pass."""
    import torch
    from paper_2303_01760_gb300 import hsm

    rng = np.random.default_rng(11)
    rows = 128 * 1000 + 37
    Xn = rng.uniform(-1.0, 1.0, size=(rows, 24))
    mlp = hsm.MLP(24, H, L, 36, seed=9)
    P = _oracle_params(mlp)
    out = mlp.predict(torch.from_numpy(Xn.astype(np.float32)).cuda()).double().cpu().numpy()
    sample = np.r_[np.arange(0, 300), rng.choice(rows, 3000, replace=False), np.arange(rows - 200, rows)]
    out_ref, _, _ = ol.forward(P, Xn[sample].astype(np.float32).astype(np.float64))
    scale = np.abs(out_ref).max()
    assert np.abs(out[sample] - out_ref).max() <= TOL_BF16_FWD * scale
    mlp.close()
