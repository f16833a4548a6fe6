"""Shared helpers for the GPU parity tests (CUDA path vs the CPU oracle)."""
import numpy as np


def to_dev(ns):
    import torch

    d = torch.device("cuda:0")
    return dict(
        spacing=None if ns.spacing is None else torch.from_numpy(np.ascontiguousarray(ns.spacing)).to(d),
        coords=torch.from_numpy(np.ascontiguousarray(ns.coords)).to(d),
        is_regular=torch.from_numpy(np.ascontiguousarray(ns.is_regular)).to(d),
        is_boundary=torch.from_numpy(np.ascontiguousarray(ns.is_boundary)).to(d),
        bc=torch.from_numpy(np.ascontiguousarray(ns.bc)).to(d),
        T_bc=torch.from_numpy(np.ascontiguousarray(ns.T_bc)).to(d),
        normals=torch.from_numpy(np.ascontiguousarray(ns.normals)).to(d),
    )


def make_plan(ns, m=2, n=0, op_mask=None, prec=0, node_status=False):
    import torch
    from paper_2303_01760_gb300 import hsm

    dv = to_dev(ns)
    plan = hsm.Plan(dv["coords"], dv["is_regular"], dv["is_boundary"], ns.h, m=m, n=n, op_mask=op_mask,
                    normals=dv["normals"], spacing=dv["spacing"])
    plan.build_stencils()
    st = torch.full((ns.N,), 77, dtype=torch.uint8, device="cuda:0") if node_status else None
    code = plan.compute_weights(prec, st, allow_singular=True)
    plan._dev = dv
    return plan, code, st


def gpu_csr(plan, op):
    rp, col, val = plan.export_csr(op)
    return rp.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()


def rows_of(rp, col, val, nodes):
    out_c, out_v = [], []
    for c in nodes:
        a, b = rp[c], rp[c + 1]
        out_c.append(col[a:b])
        out_v.append(val[a:b])
    return out_c, out_v


def rel_err_rows(w_gpu_rows, w_ref):
    """max over rows of ||w - w_ref||_inf / ||w_ref||_inf"""
    worst = 0.0
    for g, r in zip(w_gpu_rows, w_ref):
        worst = max(worst, float(np.abs(g - r).max() / np.abs(r).max()))
    return worst
