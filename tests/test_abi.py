"""The C-ABI library loads and exports every entry point include/hsm.h
declares (no GPU needed: nothing is called that touches the device)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(hsm_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def _lib():
    import __graft_entry__

    __graft_entry__.build()
    return ctypes.CDLL(os.path.join(ROOT, "paper_2303_01760_gb300", "libhsm.so"))


def test_every_declared_symbol_is_exported():
    lib = _lib()
    names = _declared()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    lib = _lib()
    lib.hsm_status_string.restype = ctypes.c_char_p
    assert lib.hsm_status_string(0) == b"ok"
    assert lib.hsm_status_string(4) == b"singular weight system"
    assert lib.hsm_status_string(99) == b"unknown status"


def test_argument_errors_need_no_device():
    """hsm_plan_create validates its arguments on the host before touching the
    device; invalid ones return HSM_EINVAL."""
    lib = _lib()
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(16)
    f = lib.hsm_plan_create
    f.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                  ctypes.c_int, ctypes.c_uint, ctypes.c_void_p]
    assert f(ctypes.byref(h), 4, 10, fake, fake, None, None, 0.1, 2, 0, 11, None) == 1
    assert f(ctypes.byref(h), 2, 10, fake, fake, None, None, -1.0, 2, 0, 11, None) == 1
    assert f(ctypes.byref(h), 2, 10, fake, fake, None, None, 0.1, 2, 6, 11, None) == 1   # n <= C(4,2)
    assert f(ctypes.byref(h), 2, 10, fake, fake, None, None, 0.1, 2, 0, 4, None) == 1    # dz in 2D
    assert f(ctypes.byref(h), 2, 10, fake, fake, None, None, 0.1, 2, 0, 11, None) == 0
    lib.hsm_plan_destroy.argtypes = [ctypes.c_void_p]
    assert lib.hsm_plan_destroy(h) == 0


def test_spacing_and_fault_hooks_validate_on_the_host():
    """hsm_plan_set_spacing and hsm_mlp_inject_fault only record their
    argument on the host: NULL handles and unknown faults give HSM_EINVAL."""
    lib = _lib()
    lib.hsm_plan_set_spacing.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.hsm_mlp_inject_fault.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.hsm_plan_set_spacing(None, None) == 1
    assert lib.hsm_mlp_inject_fault(None, 1) == 1
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(16)
    f = lib.hsm_plan_create
    f.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                  ctypes.c_int, ctypes.c_uint, ctypes.c_void_p]
    assert f(ctypes.byref(h), 2, 10, fake, fake, None, None, 0.1, 2, 0, 11, None) == 0
    assert lib.hsm_plan_set_spacing(h, fake) == 0
    assert lib.hsm_plan_set_spacing(h, None) == 0
    lib.hsm_plan_destroy.argtypes = [ctypes.c_void_p]
    assert lib.hsm_plan_destroy(h) == 0
