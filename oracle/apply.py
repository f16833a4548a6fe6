"""Operator application, Eq. 1, FP64.  Test infrastructure only.

(L u)(x_c) = sum_i w_i u(x_i) over the stencil of x_c.
"""
from __future__ import annotations

import numpy as np


def apply_group(idx, w, u):
    """idx [B, n] node ids, w [B, n] weights, u [N] -> [B]."""
    if len(idx) == 0:
        return np.zeros(0)
    return (w * u[idx]).sum(1)


def apply_all(N, st, W, u, ops):
    """Full-length outputs {op: [N]} for stencils/weights of every node.
    Nodes without a stencil in ``st`` get NaN."""
    out = {}
    for op in ops:
        o = np.full(N, np.nan)
        o[st["mon_nodes"]] = apply_group(st["mon_idx"], W["mon"][op], u)
        o[st["rbf_nodes"]] = apply_group(st["rbf_idx"], W["rbf"][op], u)
        out[op] = o
    return out


def to_csr(N, st, W, op):
    """Sparse matrix (scipy CSR) of one operator over all nodes."""
    import scipy.sparse as sp

    rows = np.concatenate([np.repeat(st["mon_nodes"], st["mon_idx"].shape[1]),
                           np.repeat(st["rbf_nodes"], st["rbf_idx"].shape[1])])
    cols = np.concatenate([st["mon_idx"].ravel(), st["rbf_idx"].ravel()])
    vals = np.concatenate([W["mon"][op].ravel(), W["rbf"][op].ravel()])
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


def wall_flux_mean(N, st, W, T, nodes, normals, scale=1.0):
    """Average Nusselt number of Section 4.1 over the given wall nodes:
    scale * mean_i |n_i . grad T(x_i)|, grad T from the first-derivative
    weights (Eq. 1), scale = L / (T_H - T_C).  normals [dim, N]."""
    dim = normals.shape[0]
    grads = apply_all(N, st, W, T, ("dx", "dy", "dz")[:dim])
    g = np.stack([grads[op][nodes] for op in ("dx", "dy", "dz")[:dim]])   # [dim, count]
    return scale * float(np.mean(np.abs((normals[:, nodes] * g).sum(0))))
