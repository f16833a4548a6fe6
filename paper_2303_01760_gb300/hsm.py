"""Thin ctypes binding of libhsm (the C ABI declared in include/hsm.h).

Argument marshalling only: every step of the method runs in the CUDA library.
Functions keep the C names; the small ``Plan`` / ``Stepper`` classes only hold
handles and turn status codes into exceptions.  Device buffers are passed as
torch CUDA tensors (their ``data_ptr()``), streams as torch streams.  There is
no CPU fallback: importing this module without the built library raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhsm.so")

HSM_DX, HSM_DY, HSM_DZ, HSM_LAP = 1, 2, 4, 8
HSM_PREC_FP64, HSM_PREC_FP32_REFINE, HSM_PREC_LEARNED = 0, 1, 2
HSM_F32, HSM_F64 = 0, 1
HSM_NODE_OK, HSM_NODE_DEMOTED, HSM_NODE_REFINE_FP64, HSM_NODE_LEARNED_SOLVE, HSM_NODE_SINGULAR = 0, 1, 2, 3, 255
HSM_NODE_REDUCED_DEGREE = 4
HSM_BC_INTERIOR, HSM_BC_T_DIRICHLET, HSM_BC_T_NEUMANN = 0, 1, 2
STATUS = {0: "HSM_OK", 1: "HSM_EINVAL", 2: "HSM_ENOMEM", 3: "HSM_ECUDA", 4: "HSM_ESINGULAR",
          5: "HSM_ENOTCONV", 6: "HSM_ETIMEOUT", 7: "HSM_EBOUNDS", 8: "HSM_ESTATE"}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libhsm.so is not built ({LIB_PATH}); run paper_2303_01760_gb300/build.py "
                      "or __graft_entry__.build()")

lib = C.CDLL(LIB_PATH)

_p = C.c_void_p
_i64 = C.c_int64


class hsm_phys(C.Structure):
    _fields_ = [("Ra", C.c_double), ("Pr", C.c_double), ("dt", C.c_double), ("T_ref", C.c_double),
                ("bc", _p), ("T_bc", _p), ("normals", _p), ("krylov_tol", C.c_double),
                ("krylov_max_it", C.c_int), ("precond", C.c_int), ("guess_order", C.c_int),
                ("apply_f32", C.c_int), ("mg_tail_from", C.c_int), ("mg_fused_from", C.c_int),
                ("mg_persistent", C.c_int), ("mg_sweeps", C.c_int), ("krylov", C.c_int)]


(HSM_OK, HSM_EINVAL, HSM_ENOMEM, HSM_ECUDA, HSM_ESINGULAR, HSM_ENOTCONV, HSM_ETIMEOUT, HSM_EBOUNDS,
 HSM_ESTATE) = range(9)
HSM_FAULT_NONE, HSM_FAULT_HOLD_MLP_LOADS, HSM_FAULT_STENCIL_INDEX = 0, 1, 2

HSM_PRECOND_AMG = 0
HSM_PRECOND_JACOBI = 1
HSM_KRYLOV_GMRES = 0
HSM_KRYLOV_BICGSTAB = 1


_SIGS = {
    "hsm_status_string": (C.c_char_p, [C.c_int]),
    "hsm_last_error": (C.c_int, [_p, C.c_char_p, C.c_size_t]),
    "hsm_plan_create": (C.c_int, [C.POINTER(_p), C.c_int, _i64, _p, _p, _p, _p, C.c_double, C.c_int,
                                  C.c_int, C.c_uint, _p]),
    "hsm_plan_build_stencils": (C.c_int, [_p]),
    "hsm_plan_compute_weights": (C.c_int, [_p, C.c_int, _p]),
    "hsm_plan_query": (C.c_int, [_p, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i64)]),
    "hsm_plan_export_csr": (C.c_int, [_p, C.c_uint, _p, _p, _p]),
    "hsm_apply": (C.c_int, [_p, C.c_uint, C.c_int, _p, _p]),
    "hsm_wall_flux_mean": (C.c_int, [_p, _p, _p, _i64, _p, C.c_double, _p]),
    "hsm_plan_condition": (C.c_int, [_p, _p]),
    "hsm_plan_set_learned_gate": (C.c_int, [_p, C.c_double, _i64]),
    "hsm_plan_learned_gate": (C.c_int, [_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(_i64)]),
    "hsm_plan_autotune": (C.c_int, [_p, C.c_char_p]),
    "hsm_plan_tuning": (C.c_int, [_p] + [C.POINTER(C.c_int)] * 7),
    "hsm_plan_set_tuning": (C.c_int, [_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
    "hsm_plan_validate": (C.c_int, [_p]),
    "hsm_plan_set_checks": (C.c_int, [_p, C.c_int]),
    "hsm_plan_inject_fault": (C.c_int, [_p, C.c_int]),
    "hsm_plan_destroy": (C.c_int, [_p]),
    "hsm_plan_profile": (C.c_int, [_p, C.POINTER(C.c_float), C.POINTER(_i64)]),
    "hsm_plan_set_timing": (C.c_int, [_p, C.c_int]),
    "hsm_plan_set_spacing": (C.c_int, [_p, _p]),
    "hsm_stepper_create": (C.c_int, [C.POINTER(_p), _p, C.POINTER(hsm_phys)]),
    "hsm_step": (C.c_int, [_p, C.c_int, _p, _p, _p, C.POINTER(C.c_int)]),
    "hsm_stepper_destroy": (C.c_int, [_p]),
    "hsm_stepper_info": (C.c_int, [_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                   C.POINTER(C.c_int), C.POINTER(C.c_int), _p, _p, C.POINTER(C.c_int),
                                   C.POINTER(C.c_float), _p, _p]),
    "hsm_rbf_weights_fp32r_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_uint, _p, _i64, _p, _i64, _p, _p,
                                                _p]),
    "hsm_mlp_create": (C.c_int, [C.POINTER(_p), C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, _p]),
    "hsm_mlp_destroy": (C.c_int, [_p]),
    "hsm_mlp_param_count": (C.c_int, [_p, C.POINTER(_i64)]),
    "hsm_mlp_get_params": (C.c_int, [_p, _p, _i64]),
    "hsm_mlp_set_params": (C.c_int, [_p, _p, _i64]),
    "hsm_mlp_grad": (C.c_int, [_p, _p, _p, _i64, _p, C.POINTER(C.c_float)]),
    "hsm_mlp_train": (C.c_int, [_p, _p, _p, _i64, C.c_int, C.c_int, C.c_float, C.c_uint64, _p]),
    "hsm_mlp_predict": (C.c_int, [_p, _p, _i64, _p]),
    "hsm_mlp_inject_fault": (C.c_int, [_p, C.c_int]),
    "hsm_mlp_attach": (C.c_int, [_p, _p]),
    "hsm_plan_learned_data": (C.c_int, [_p, _p, _p, C.POINTER(_i64)]),
    "hsm_probe_fp64_peak": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_float), _p]),
    "hsm_eval_helper": (C.c_int, [C.c_int, _p, _p, _i64, _p]),
}
HSM_HELPER_RECIP, HSM_HELPER_SQRT_NR1, HSM_HELPER_SQRT_GS, HSM_HELPER_ERF_AS, HSM_HELPER_GELU = range(5)
HSM_NOALLOC_MAX_SYSTEMS = 1 << 20
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name, None)
    if _f is not None:
        _f.restype = _res
        _f.argtypes = _args
        globals()[_name] = _f


class HsmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def last_error(handle=None) -> str:
    buf = C.create_string_buffer(1024)
    lib.hsm_last_error(handle, buf, 1024)
    return buf.value.decode(errors="replace")


def check(code, handle=None):
    if code != 0:
        raise HsmError(code, last_error(handle))
    return code


def ptr(t):
    """Device pointer of a torch tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libhsm needs CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("libhsm needs contiguous tensors")
    return C.c_void_p(t.data_ptr())


def stream_handle(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def op_list(mask, dim):
    names = []
    for b, nm in ((1, "dx"), (2, "dy"), (4, "dz"), (8, "lap")):
        if mask & b:
            names.append(nm)
    return names


def _binom(a, b):
    from math import comb

    return comb(a, b)


class MLP:
    """Owns an hsm_mlp (the learned weight predictor)."""

    def __init__(self, n_in=24, hidden=256, layers=3, n_out=36, seed=1, stream=None):
        h_ = C.c_void_p()
        check(lib.hsm_mlp_create(C.byref(h_), int(n_in), int(hidden), int(layers), int(n_out), int(seed),
                                 stream_handle(stream)))
        self.h = h_
        self.n_in, self.n_out = n_in, n_out

    def param_count(self):
        c = _i64()
        check(lib.hsm_mlp_param_count(self.h, C.byref(c)))
        return c.value

    def get_params(self):
        import numpy as np

        buf = np.empty(self.param_count(), dtype=np.float32)
        check(lib.hsm_mlp_get_params(self.h, buf.ctypes.data_as(C.c_void_p), buf.size))
        return buf

    def set_params(self, flat):
        import numpy as np

        buf = np.ascontiguousarray(flat, dtype=np.float32)
        check(lib.hsm_mlp_set_params(self.h, buf.ctypes.data_as(C.c_void_p), buf.size))

    def grad(self, X, Y):
        import numpy as np

        g = np.empty(self.param_count(), dtype=np.float32)
        loss = C.c_float()
        check(lib.hsm_mlp_grad(self.h, ptr(X), ptr(Y), X.shape[0], g.ctypes.data_as(C.c_void_p), C.byref(loss)))
        return float(loss.value), g

    def train(self, X, Y, steps, batch=1024, lr=1e-3, seed=7):
        import numpy as np

        log = np.empty(max(steps, 1), dtype=np.float32)
        check(lib.hsm_mlp_train(self.h, ptr(X), ptr(Y), X.shape[0], int(steps), int(batch), float(lr), int(seed),
                                log.ctypes.data_as(C.c_void_p)))
        return log[:steps]

    def inject_fault(self, fault=HSM_FAULT_HOLD_MLP_LOADS):
        """Failure-path test hook: the next fused forward pass issues no loads,
        so its bounded waits expire and predict raises HSM_ETIMEOUT."""
        check(lib.hsm_mlp_inject_fault(self.h, int(fault)))

    def predict(self, X):
        import torch

        Y = torch.empty((X.shape[0], self.n_out), dtype=torch.float32, device=X.device)
        check(lib.hsm_mlp_predict(self.h, ptr(X), X.shape[0], ptr(Y)))
        return Y

    def close(self):
        if self.h:
            lib.hsm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def unpack_params(flat, n_in, hidden, layers, n_out):
    """Packed parameter vector -> [(W [out, in], b [out]), ...] (float64)."""
    import numpy as np

    dims = [n_in] + [hidden] * layers + [n_out]
    out, k = [], 0
    for a, b in zip(dims[:-1], dims[1:]):
        W = np.asarray(flat[k:k + a * b], dtype=np.float64).reshape(b, a)
        k += a * b
        bb = np.asarray(flat[k:k + b], dtype=np.float64)
        k += b
        out.append((W, bb))
    return out


class Plan:
    """Owns an hsm_plan.  ``coords`` (f64 [dim, N]), ``is_regular`` and
    ``is_boundary`` (u8 [N]) and ``normals`` (f64 [dim, N]) are CUDA tensors
    that must outlive the plan."""

    def __init__(self, coords, is_regular, is_boundary, h, m=2, n=0, op_mask=None, stream=None, normals=None,
                 spacing=None):
        dim, N = coords.shape
        if op_mask is None:
            op_mask = HSM_DX | HSM_DY | HSM_LAP | (HSM_DZ if dim == 3 else 0)
        self.dim, self.N, self.op_mask = dim, N, op_mask
        self.n = n if n else 2 * _binom(m + dim, m)
        self._keep = (coords, is_regular, is_boundary, normals, spacing)
        h_ = C.c_void_p()
        check(lib.hsm_plan_create(C.byref(h_), dim, N, ptr(coords), ptr(is_regular), ptr(is_boundary),
                                  ptr(normals), float(h), int(m), int(n), int(op_mask), stream_handle(stream)))
        self.h = h_
        if spacing is not None:
            check(lib.hsm_plan_set_spacing(self.h, ptr(spacing)), self.h)

    def build_stencils(self):
        check(lib.hsm_plan_build_stencils(self.h), self.h)
        return self

    def set_spacing(self, spacing):
        """Local internodal distance h(x_i) (f64 CUDA [N], or None for h_regular)
        of an h-refined set; takes effect at the next build_stencils."""
        check(lib.hsm_plan_set_spacing(self.h, ptr(spacing)), self.h)
        self._keep = self._keep[:4] + (spacing,)
        return self

    def compute_weights(self, prec=HSM_PREC_FP64, node_status=None, allow_singular=False):
        code = lib.hsm_plan_compute_weights(self.h, int(prec), ptr(node_status))
        if code == 4 and allow_singular:
            return code
        check(code, self.h)
        return code

    def query(self):
        a, b, c, d = _i64(), _i64(), _i64(), _i64()
        check(lib.hsm_plan_query(self.h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)), self.h)
        return dict(nnz_per_op=a.value, n_mon=b.value, n_demoted=c.value, n_fallback=d.value)

    def export_csr(self, op):
        import torch

        q = self.query()
        dev = self._keep[0].device
        rp = torch.empty(self.N + 1, dtype=torch.int64, device=dev)
        col = torch.empty(q["nnz_per_op"], dtype=torch.int32, device=dev)
        val = torch.empty(q["nnz_per_op"], dtype=torch.float64, device=dev)
        check(lib.hsm_plan_export_csr(self.h, int(op), ptr(rp), ptr(col), ptr(val)), self.h)
        return rp, col, val

    def apply(self, u, op_mask=None, out=None):
        import torch

        op_mask = self.op_mask if op_mask is None else op_mask
        k = bin(op_mask).count("1")
        if out is None:
            out = torch.empty((k, self.N), dtype=torch.float64, device=u.device)
        dt = HSM_F64 if u.dtype == torch.float64 else HSM_F32
        if u.dtype not in (torch.float64, torch.float32):
            raise ValueError("u must be float32 or float64")
        check(lib.hsm_apply(self.h, int(op_mask), dt, ptr(u), ptr(out)), self.h)
        return out

    def condition(self, out=None):
        """kappa_2 of every node's weight system (Section 2.1), f64 CUDA [N]."""
        import torch

        if out is None:
            out = torch.empty(self.N, dtype=torch.float64, device=self._keep[0].device)
        check(lib.hsm_plan_condition(self.h, ptr(out)), self.h)
        return out

    def wall_flux_mean(self, T, nodes, normals, scale=1.0, out=None):
        """scale * mean over ``nodes`` of |n . grad T| (the average Nusselt
        number of Section 4.1); a one-element f64 CUDA tensor, not synchronised."""
        import torch

        if out is None:
            out = torch.empty(1, dtype=torch.float64, device=T.device)
        nodes = nodes.to(torch.int32).contiguous()
        check(lib.hsm_wall_flux_mean(self.h, ptr(T), ptr(nodes), int(nodes.numel()), ptr(normals), float(scale),
                                     ptr(out)), self.h)
        self._flux_keep = nodes
        return out

    def set_timing(self, enable=True):
        check(lib.hsm_plan_set_timing(self.h, 1 if enable else 0), self.h)

    def profile(self):
        """(per-phase device ms [stencils, MON, RBF-FD, apply], kernels launched)"""
        ms = (C.c_float * 4)()
        n = _i64()
        check(lib.hsm_plan_profile(self.h, ms, C.byref(n)), self.h)
        return list(ms), n.value

    def learned_data(self, labels=True):
        """(X [count, d*n], Y [count, nops*n] or None) of the interior RBF-FD
        stencils, float32 CUDA tensors."""
        import torch

        cnt = _i64()
        check(lib.hsm_plan_learned_data(self.h, None, None, C.byref(cnt)), self.h)
        dev = self._keep[0].device
        X = Y = None
        if cnt.value:
            nops = bin(self.op_mask).count("1")
            n = self.n
            X = torch.empty((cnt.value, self.dim * n), dtype=torch.float32, device=dev)
            Y = torch.empty((cnt.value, nops * n), dtype=torch.float32, device=dev) if labels else None
            check(lib.hsm_plan_learned_data(self.h, ptr(X), ptr(Y), C.byref(cnt)), self.h)
        return X, Y

    def set_learned_gate(self, tol=1e-3, samples=512):
        """Batch validation of the learned weights (samples = 0 turns it off)."""
        check(lib.hsm_plan_set_learned_gate(self.h, float(tol), int(samples)), self.h)

    def learned_gate(self):
        """(mean relative error of the validated samples, batch fell back,
        accepted samples the error averages)."""
        e, f, a = C.c_double(), C.c_int(), _i64()
        check(lib.hsm_plan_learned_gate(self.h, C.byref(e), C.byref(f), C.byref(a)), self.h)
        return e.value, bool(f.value), a.value

    def attach(self, mlp):
        check(lib.hsm_mlp_attach(self.h, mlp.h if mlp is not None else None), self.h)
        self._mlp = mlp

    def autotune(self, cache_path=None):
        check(lib.hsm_plan_autotune(self.h, cache_path.encode() if cache_path else None), self.h)

    def validate(self):
        """Status of the stencil-table scan (HSM_OK or HSM_EBOUNDS); not raised."""
        return lib.hsm_plan_validate(self.h)

    def set_checks(self, enable=True):
        check(lib.hsm_plan_set_checks(self.h, int(bool(enable))), self.h)

    def inject_stencil_fault(self):
        check(lib.hsm_plan_inject_fault(self.h, HSM_FAULT_STENCIL_INDEX), self.h)

    def set_tuning(self, knn_qt=1, rbf_lanes=8, rbf_lanes32=8, apply_threads=256, arrange=0, chunks=1):
        """arrange: 0 MON weights in the build and one RBF-FD launch, 1 one
        grouped launch, 2 both groups in the build (RBF-FD in `chunks` chunks
        beside the kNN search)."""
        check(lib.hsm_plan_set_tuning(self.h, int(knn_qt), int(rbf_lanes), int(rbf_lanes32), int(apply_threads),
                                      int(arrange), int(chunks)), self.h)

    def tuning(self):
        v = [C.c_int() for _ in range(7)]
        check(lib.hsm_plan_tuning(self.h, *[C.byref(x) for x in v]), self.h)
        return dict(zip(("knn_qt", "rbf_lanes", "rbf_lanes32", "apply_threads", "arrange", "chunks", "tuned"),
                        [x.value for x in v]))

    def close(self):
        if self.h:
            lib.hsm_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Stepper:
    """Owns an hsm_stepper on a plan (Section 3 explicit Boussinesq step)."""

    def __init__(self, plan, Ra, Pr, dt, T_ref, bc, T_bc, normals, krylov_tol=1e-12, krylov_max_it=2000,
                 precond=HSM_PRECOND_AMG, guess_order=0, apply_f32=False, mg_tail_from=0, mg_fused_from=0,
                 mg_persistent=0, mg_sweeps=0, krylov=0):
        self.plan = plan
        self._keep = (bc, T_bc, normals)
        self.phys = hsm_phys(float(Ra), float(Pr), float(dt), float(T_ref), ptr(bc).value, ptr(T_bc).value,
                             ptr(normals).value, float(krylov_tol), int(krylov_max_it), int(precond),
                             int(guess_order), int(bool(apply_f32)), int(mg_tail_from), int(mg_fused_from),
                             int(mg_persistent), int(mg_sweeps), int(krylov))
        h_ = C.c_void_p()
        check(lib.hsm_stepper_create(C.byref(h_), plan.h, C.byref(self.phys)), plan.h)
        self.h = h_

    def info(self):
        a, b, c, f, d, pe = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
        ms, fms, pms = (C.c_float * 16)(), (C.c_float * 16)(), C.c_float()
        rows, ents = (C.c_int64 * 16)(), (C.c_int64 * 16)()
        check(lib.hsm_stepper_info(self.h, C.byref(a), C.byref(b), C.byref(c), C.byref(f), C.byref(d), ms, fms,
                                   C.byref(pe), C.byref(pms), rows, ents))
        n = max(a.value, 1)
        return dict(mg_levels=a.value, mg_tail_level=b.value, mg_tail_ctas=c.value, mg_fused_level=f.value,
                    kernels_per_iter=d.value, tail_ms_10_cycles=[round(x, 4) for x in ms[:n]],
                    fused_ms_10_cycles=[round(x, 4) for x in fms[:n]], mg_persistent=pe.value,
                    persistent_ms_10_cycles=round(pms.value, 4), level_rows=list(rows[:a.value]),
                    level_entries=list(ents[:a.value]))

    def step(self, v, T, p, n_steps=1, allow_notconv=False):
        iters = (C.c_int * max(1, n_steps))()
        code = lib.hsm_step(self.h, int(n_steps), ptr(v), ptr(T), ptr(p), iters)
        if not (code == 5 and allow_notconv):
            check(code, self.plan.h)
        return list(iters)[:n_steps], code

    def close(self):
        if self.h:
            lib.hsm_stepper_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rbf_weights_fp32r_noalloc(dim, m, n, op_mask, coords, stencils, weights, node_status=None, stream=None):
    """Allocation-free RBF-FD weights for caller-supplied stencils
    (``stencils`` int32 [n, count], row 0 = centres; ``weights`` f64
    [nops, n, count] is written).  For callers that must not allocate device
    memory while they run; the library keeps its scratch in a fixed static
    device array.  Returns the status code."""
    return lib.hsm_rbf_weights_fp32r_noalloc(int(dim), int(m), int(n), int(op_mask), ptr(coords),
                                             int(coords.shape[1]), ptr(stencils), int(stencils.shape[1]),
                                             ptr(weights), ptr(node_status), stream_handle(stream))


def probe_fp64_peak(stream=None):
    """Measured FP64 FMA throughput of the current device: (GFLOP/s, ms)."""
    g, ms = C.c_double(), C.c_float()
    check(lib.hsm_probe_fp64_peak(C.byref(g), C.byref(ms), stream_handle(stream)))
    return g.value, ms.value


def eval_helper(fn, x, stream=None):
    """One of the HSM_HELPER_* device math helpers applied elementwise to the
    f64 CUDA tensor ``x``; returns a new f64 tensor."""
    import torch

    y = torch.empty_like(x)
    check(lib.hsm_eval_helper(int(fn), ptr(x), ptr(y), int(x.numel()), stream_handle(stream)))
    return y
