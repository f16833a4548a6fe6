"""Learned stencil weights: FP64 MLP and the exact consistency projection.

Test infrastructure only (see the package docstring).  The paper has no
learned component; this follows the specification of the learned weight
predictor (an MLP from the normalised neighbour offsets of a scattered stencil
to its operator weights, trained on weights of the plain solver, its output
projected exactly onto the monomial-reproduction constraints up to degree m,
the direct solve as fallback).

Definitions used by both the oracle and the tests:

* Canonical frame (2D): an orthogonal Q per stencil that turns the offset of
  the nearest neighbour (stencil entry 1) onto +x and, by a reflection if
  needed, puts entry 2 in the upper half plane.  The Laplacian is invariant
  and the derivative pair transforms as a vector, so the network only has to
  learn stencils in one orientation.
* Features: the n scaled offsets Q (x_i - x_c)/s, s = max |x_i - x_c|, in
  stencil order, flattened as (xi_1x, xi_1y, xi_2x, ...) -- 2n values.
* Labels: the weights in the scaled canonical variable: Q (s w_dx, s w_dy)
  per node for the derivatives, s^2 w for the Laplacian, flattened op-major
  [op][node] -- 3n values.  Predictions are turned back with Q^T.
* MLP: Linear(2n, H) -> GELU -> (Linear(H, H) -> GELU) x (L-1) ->
  Linear(H, 3n); GELU(x) = x Phi(x) with Phi the standard normal CDF.
  Loss = mean over batch and outputs of (y - t)^2.
* Projection (Eq. 1 enforced for the monomials of degree <= m, Section 2):
      w = w_hat + P (P^T P)^{-1} (l_p - P^T w_hat)
  per operator, with P_ij = p_j(xi_i) and l_p = L p_j at the centre: the
  minimum-Euclidean-norm correction that makes the weights reproduce every
  monomial of degree <= m exactly.
* Fallback to the direct solve when the post-projection residual exceeds
  1e-10 (scaled units), or when the relative pre-projection residual
  |P^T w_hat - l_p| / |l_p| exceeds tau_ood = 1.5 (a prediction that far from
  consistent is treated as out of distribution).

Pins: GELU by closed-form values of the normal CDF; the forward pass by a
hand-computed 2-2-1 network; the gradients by finite differences of the loss;
Adam by its bias-corrected first step; the projection by its defining
properties (constraints met, correction in range(P), minimum norm, exact
weights are a fixed point).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from . import weights as ow

TAU_OOD = 1.5
POST_TOL = 1e-10


def canonical_frame(xi):
    """Q [B, 2, 2] for scaled 2D offsets xi [B, n, 2]."""
    v = xi[:, 1, :]
    r = np.sqrt((v ** 2).sum(1))
    c, sn = v[:, 0] / r, v[:, 1] / r
    Q = np.stack([np.stack([c, sn], 1), np.stack([-sn, c], 1)], 1)
    y2 = np.einsum("bj,bj->b", Q[:, 1, :], xi[:, 2, :])
    Q[y2 < 0, 1, :] *= -1.0
    return Q


def features_labels(coords, stencil, W=None):
    """X [B, 2n] canonical scaled offsets; Y [B, 3n] canonical scaled
    weights (if W given); s [B]; Q [B, 2, 2]."""
    xi, s = ow._scaled_offsets(coords, stencil)
    B, n, dim = xi.shape
    Q = canonical_frame(xi)
    X = np.einsum("bij,bnj->bni", Q, xi).reshape(B, n * dim)
    if W is None:
        return X, None, s, Q
    wd = np.stack([W["dx"] * s[:, None], W["dy"] * s[:, None]], 2)       # [B, n, 2]
    wdc = np.einsum("bij,bnj->bni", Q, wd)
    Y = np.concatenate([wdc[:, :, 0], wdc[:, :, 1], W["lap"] * s[:, None] ** 2], 1)
    return X, Y, s, Q


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def init_params(n_in, hidden, layers, n_out, seed=0):
    """He-uniform style initialisation (uniform +-sqrt(6/fan_in)/2), zero bias."""
    rng = np.random.default_rng(seed)
    dims = [n_in] + [hidden] * layers + [n_out]
    P = []
    for a, b in zip(dims[:-1], dims[1:]):
        lim = math.sqrt(6.0 / a) * 0.5
        P.append((rng.uniform(-lim, lim, (b, a)), np.zeros(b)))
    return P


def forward(P, X):
    """Returns output and the list of pre-activations / activations."""
    acts = [X]
    pre = []
    h = X
    for li, (Wt, b) in enumerate(P):
        z = h @ Wt.T + b
        pre.append(z)
        h = gelu(z) if li < len(P) - 1 else z
        acts.append(h)
    return h, pre, acts


def loss_and_grad(P, X, Y):
    out, pre, acts = forward(P, X)
    B, O = out.shape
    diff = out - Y
    loss = float((diff ** 2).mean())
    g = 2.0 * diff / (B * O)
    grads = [None] * len(P)
    for li in range(len(P) - 1, -1, -1):
        Wt, b = P[li]
        grads[li] = (g.T @ acts[li], g.sum(0))
        if li > 0:
            g = (g @ Wt) * gelu_grad(pre[li - 1])
    return loss, grads


def adam_step(P, grads, state, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) of all parameters in place."""
    if state is None:
        state = [[(np.zeros_like(W), np.zeros_like(W)), (np.zeros_like(b), np.zeros_like(b))] for W, b in P]
    newP = []
    for li, ((W, b), (gW, gb)) in enumerate(zip(P, grads)):
        out = []
        for k, (p, gp) in enumerate(((W, gW), (b, gb))):
            m, v = state[li][k]
            m = beta1 * m + (1 - beta1) * gp
            v = beta2 * v + (1 - beta2) * gp * gp
            state[li][k] = (m, v)
            mh = m / (1 - beta1 ** t)
            vh = v / (1 - beta2 ** t)
            out.append(p - lr * mh / (np.sqrt(vh) + eps))
        newP.append(tuple(out))
    return newP, state


def constraint_system(xi, m, ops):
    """P [B, n, Mp] and l_p [B, Mp, nops] at the scaled offsets xi [B, n, dim]."""
    dim = xi.shape[2]
    exps = ow.monomial_exponents(dim, m)
    Pm = ow.eval_monomials(exps, xi)
    lp = np.stack([ow.L_monomials_at_center(exps, op, dim) for op in ops], -1)
    return Pm, np.broadcast_to(lp, (xi.shape[0],) + lp.shape).copy()


def project(w_hat, Pm, lp):
    """w_hat [B, n, nops] -> projected w and the pre-projection relative residual."""
    r = lp - np.einsum("bnj,bno->bjo", Pm, w_hat)
    G = np.einsum("bnj,bnk->bjk", Pm, Pm)
    c = np.linalg.solve(G, r)
    w = w_hat + np.einsum("bnj,bjo->bno", Pm, c)
    pre = np.linalg.norm(r, axis=1) / np.maximum(np.linalg.norm(lp, axis=1), 1e-300)
    return w, pre


def post_residual(w, Pm, lp):
    return np.abs(np.einsum("bnj,bno->bjo", Pm, w) - lp).max(axis=(1, 2))


def learned_weights(coords, stencil, m, out_scaled, ops=("dx", "dy", "lap")):
    """Projection and fallback decision for MLP outputs ``out_scaled`` [B, 3n]
    (scaled weights).  Returns ({op: w [B, n]} physical weights, accept [B])."""
    xi, s = ow._scaled_offsets(coords, stencil)
    B, n, dim = xi.shape
    w_hat = out_scaled.reshape(B, len(ops), n).transpose(0, 2, 1).copy()
    Q = canonical_frame(xi)
    w_hat[:, :, :2] = np.einsum("bji,bnj->bni", Q, w_hat[:, :, :2])   # Q^T per node
    Pm, lp = constraint_system(xi, m, ops)
    w, pre = project(w_hat, Pm, lp)
    post = post_residual(w, Pm, lp)
    accept = (pre.max(1) <= TAU_OOD) & (post <= POST_TOL)
    out = {}
    for k, op in enumerate(ops):
        p = 2 if op == "lap" else 1
        out[op] = w[:, :, k] / s[:, None] ** p
    return out, accept
