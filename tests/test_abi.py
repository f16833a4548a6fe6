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


def _declarations():
    """{name: [parameter type strings]} of every function in include/*.h."""
    out = {}
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        for m in re.finditer(r"\b(hsm_[a-z0-9_]+)\s*\(([^;{}]*?)\)\s*;", txt):
            params = [p.strip() for p in m.group(2).split(",")]
            out[m.group(1)] = [] if params in ([""], ["void"]) else params
    return out


def _kind_of_c(param, handles, enums):
    """Broad kind of a C parameter: the type without its name."""
    t = re.sub(r"\b(const|struct|unsigned\s+char)\b", lambda m: "uchar" if "char" in m.group(0) else "", param)
    if "*" in t or "[" in t:
        return "ptr"
    words = t.split()
    base = " ".join(words[:-1]) if len(words) > 1 else words[0]
    if base in handles:
        return "ptr"
    if base in enums or base in ("int", "int32_t"):
        return "i32"
    if base in ("unsigned", "unsigned int", "uint32_t"):
        return "u32"
    if base in ("int64_t", "long long"):
        return "i64"
    if base in ("uint64_t", "size_t"):
        return "u64"
    return {"double": "f64", "float": "f32"}.get(base, "?" + base)


def _kind_of_ctypes(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and isinstance(t._type_, type):
        return "ptr"
    size = ctypes.sizeof(t)
    if t in (ctypes.c_double,):
        return "f64"
    if t in (ctypes.c_float,):
        return "f32"
    signed = t(-1).value < 0
    return {(4, True): "i32", (4, False): "u32", (8, True): "i64", (8, False): "u64"}[(size, signed)]


def test_binding_prototypes_match_the_header():
    """Every ctypes prototype of the Python binding has the parameter count
    and the broad parameter types (pointer, 32/64-bit signed/unsigned
    integer, float, double) that include/hsm.h declares, so a signature
    change on one side cannot go unnoticed until a GPU run."""
    import sys

    sys.path.insert(0, ROOT)
    from paper_2303_01760_gb300 import hsm

    header = open(os.path.join(ROOT, "include", "hsm.h")).read()
    handles = set(re.findall(r"typedef\s+struct\s+\w+\s*\*\s*(\w+)\s*;", header))
    enums = set(re.findall(r"}\s*(hsm_\w+)\s*;", header)) - handles
    decl = _declarations()
    assert len(decl) >= 30
    checked = 0
    for name, (_, args) in hsm._SIGS.items():
        assert name in decl, name
        c_kinds = [_kind_of_c(p, handles, enums) for p in decl[name]]
        py_kinds = [_kind_of_ctypes(a) for a in args]
        assert c_kinds == py_kinds, (name, c_kinds, py_kinds)
        checked += 1
    assert checked == len(hsm._SIGS) >= 30
