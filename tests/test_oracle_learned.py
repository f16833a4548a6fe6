"""Pins for the oracle's learned-weight pieces: GELU, MLP gradients, Adam,
and the consistency projection (its defining properties)."""
import numpy as np
import pytest

from oracle import learned as ol
from oracle import stencils as ost
from oracle import weights as ow
from paper_2303_01760_gb300 import nodesets


def test_gelu_standard_normal_values():
    # GELU(x) = x Phi(x); Phi(1) = 0.8413447460685429, Phi(2) = 0.9772498680518208
    assert abs(ol.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    assert abs(ol.gelu(np.array(-1.0)) + 0.15865525393145707) < 1e-15
    assert abs(ol.gelu(np.array(2.0)) - 2 * 0.9772498680518208) < 1e-15
    assert ol.gelu(np.array(0.0)) == 0.0
    x = np.linspace(-4, 4, 41)
    h = 1e-6
    fd = (ol.gelu(x + h) - ol.gelu(x - h)) / (2 * h)
    assert np.abs(fd - ol.gelu_grad(x)).max() < 1e-8


def test_mlp_gradients_against_finite_differences():
    rng = np.random.default_rng(0)
    P = ol.init_params(6, 7, 2, 4, seed=1)
    P = [(W + 0.1 * rng.normal(size=W.shape), b + 0.1 * rng.normal(size=b.shape)) for W, b in P]
    X = rng.normal(size=(9, 6))
    Y = rng.normal(size=(9, 4))
    loss, grads = ol.loss_and_grad(P, X, Y)
    eps = 1e-6
    for li in range(len(P)):
        for k in range(2):
            arr = P[li][k]
            for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(4)]:
                Pp = [(W.copy(), b.copy()) for W, b in P]
                Pm = [(W.copy(), b.copy()) for W, b in P]
                Pp[li][k][idx] += eps
                Pm[li][k][idx] -= eps
                fd = (ol.loss_and_grad(Pp, X, Y)[0] - ol.loss_and_grad(Pm, X, Y)[0]) / (2 * eps)
                assert abs(fd - grads[li][k][idx]) <= 1e-7 + 1e-5 * abs(fd)


def test_adam_first_step_moves_by_learning_rate():
    """Kingma and Ba: the bias-corrected first step is lr * g / (|g| + eps)."""
    P = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    g = [(np.array([[0.5, -3.0]]), np.array([1e-3]))]
    P2, _ = ol.adam_step(P, g, None, lr=0.1, t=1)
    assert np.allclose(P2[0][0], [[0.9, -1.9]], atol=1e-6)
    assert np.allclose(P2[0][1], [0.4], atol=1e-4)


def _stencils(n_set=30, seed=nodesets.SEED_BASE + 40):
    ns = nodesets.square_all_scattered(n=n_set, seed=seed, jitter=0.2)
    inner = np.flatnonzero((ns.is_boundary == 0) & (np.minimum(ns.coords, 1 - ns.coords).min(0) > 0.15))
    st = ost.knn_bruteforce(ns.coords, inner[:200], 12)
    return ns, st


def test_projection_fixed_point_and_constraints():
    ns, st = _stencils()
    W = ow.rbffd_weights(ns.coords, st, 2)
    X, Y, s, Q = ol.features_labels(ns.coords, st, W)
    w_exact, acc = ol.learned_weights(ns.coords, st, 2, Y)
    assert acc.all()
    for op in ("dx", "dy", "lap"):
        assert np.abs(w_exact[op] - W[op]).max() <= 1e-10 * np.abs(W[op]).max()
    # random perturbation: projected weights meet every constraint, the
    # correction lies in range(P), and it is the shortest such correction
    rng = np.random.default_rng(3)
    xi, _ = ow._scaled_offsets(ns.coords, st)
    Pm, lp = ol.constraint_system(xi, 2, ("dx", "dy", "lap"))
    w_hat = np.stack([W["dx"] * s[:, None], W["dy"] * s[:, None], W["lap"] * s[:, None] ** 2], 2)
    w_hat = w_hat + 0.05 * rng.normal(size=(len(st), 12, 3))
    w, pre = ol.project(w_hat, Pm, lp)
    assert ol.post_residual(w, Pm, lp).max() <= 1e-12
    assert pre.max() > 0
    for b in range(5):
        for o in range(3):
            d = w[b, :, o] - w_hat[b, :, o]
            c, *_ = np.linalg.lstsq(Pm[b], d, rcond=None)
            assert np.abs(Pm[b] @ c - d).max() <= 1e-12 * max(1.0, np.abs(d).max())
            _, _, vt = np.linalg.svd(Pm[b].T)
            z = vt[6:].T @ rng.normal(size=6)
            assert np.linalg.norm(w[b, :, o] + 0.1 * z - w_hat[b, :, o]) > np.linalg.norm(d)


def test_projection_rejects_out_of_distribution_predictions():
    ns, st = _stencils()
    W = ow.rbffd_weights(ns.coords, st, 2)
    X, Y, s, Q = ol.features_labels(ns.coords, st, W)
    bad = Y.copy()
    bad[:10] = 50.0  # grossly wrong predictions: far outside the constraint set
    _, acc = ol.learned_weights(ns.coords, st, 2, bad)
    assert not acc[:10].any() and acc[10:].all()


def test_training_reduces_loss():
    ns, st = _stencils()
    W = ow.rbffd_weights(ns.coords, st, 2)
    X, Y, _, _ = ol.features_labels(ns.coords, st, W)
    P = ol.init_params(24, 32, 2, 36, seed=5)
    l0 = ol.loss_and_grad(P, X, Y)[0]
    state = None
    for t in range(1, 301):
        loss, g = ol.loss_and_grad(P, X, Y)
        P, state = ol.adam_step(P, g, state, lr=3e-3, t=t)
    assert ol.loss_and_grad(P, X, Y)[0] < 0.1 * l0


def test_canonical_frame_is_orthogonal_and_canonical():
    ns, st = _stencils()
    W = ow.rbffd_weights(ns.coords, st, 2)
    X, Y, s, Q = ol.features_labels(ns.coords, st, W)
    assert np.allclose(np.einsum("bij,bkj->bik", Q, Q), np.eye(2)[None], atol=1e-14)
    Xr = X.reshape(len(st), 12, 2)
    assert np.all(np.abs(Xr[:, 1, 1]) <= 1e-14) and np.all(Xr[:, 1, 0] > 0) and np.all(Xr[:, 2, 1] >= 0)
    # the derivative weights are a vector field: the canonical labels are the
    # weights of the rotated stencil itself
    xi_c = Xr
    coords_c = np.concatenate([xi_c[b].T for b in range(3)], 1)
    st_c = np.arange(36).reshape(3, 12)
    Wc = ow.rbffd_weights(coords_c, st_c, 2)
    for b in range(3):
        assert np.allclose(Wc["dx"][b], Y[b, :12], atol=1e-9 * np.abs(Y[b]).max())
        assert np.allclose(Wc["dy"][b], Y[b, 12:24], atol=1e-9 * np.abs(Y[b]).max())
        assert np.allclose(Wc["lap"][b], Y[b, 24:], atol=1e-9 * np.abs(Y[b]).max())


def test_mlp_forward_hand_computed():
    """A 2-2-1 network with hand-chosen weights: the output is fixed by the
    standard normal CDF values Phi(1) and Phi(2) alone."""
    P = [(np.eye(2), np.zeros(2)), (np.array([[1.0, -3.0]]), np.array([0.5]))]
    out, pre, _ = ol.forward(P, np.array([[1.0, 2.0], [-1.0, 0.0]]))
    phi1, phi2 = 0.8413447460685429, 0.9772498680518208
    assert abs(out[0, 0] - (phi1 - 3.0 * 2.0 * phi2 + 0.5)) < 1e-14
    # gelu(-1) = -(1 - Phi(1)), gelu(0) = 0
    assert abs(out[1, 0] - (-(1.0 - phi1) + 0.5)) < 1e-14
    assert np.array_equal(pre[0], np.array([[1.0, 2.0], [-1.0, 0.0]]))


def test_bf16_inputs_alone_move_the_weights_beyond_the_learned_tolerance():
    """The learned predictor's tensor-core layers take bf16 inputs (8-bit
    significand).  Rounding the scaled offsets of interior scattered stencils
    to bf16 and solving exactly moves the weights by about 1.4e-3 relative
    (median; mean about 1.6e-3) on a Poisson-disk set: above the 1e-3 gate of
    the learned path, before any approximation error of the network.  A
    network whose first layer reads bf16 offsets cannot meet that gate on
    average, however well trained."""
    torch = pytest.importorskip("torch")
    ns = nodesets.square_all_scattered(n=60, seed=nodesets.SEED_BASE + 700)
    st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, 12, normals=ns.normals)
    idx = st["rbf_idx"][ns.is_boundary[st["rbf_nodes"]] == 0][:1500]
    xi, _ = ow._scaled_offsets(ns.coords, idx)

    def solve(x):
        M, rhs = ow.rbffd_system(x, 2, ow.ops_for(2))
        return np.linalg.solve(M, rhs)[:, :12, :]

    w = solve(xi)
    xb = torch.from_numpy(xi).to(torch.bfloat16).to(torch.float64).numpy()
    rel = np.abs(solve(xb) - w).max((1, 2)) / np.abs(w).max((1, 2))
    assert np.abs(xb - xi).max() <= 2.0 ** -9 * np.abs(xi).max()   # bf16 rounding, nothing more
    assert rel.mean() > 1e-3 and np.median(rel) > 7e-4
