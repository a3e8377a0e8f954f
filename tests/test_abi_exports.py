"""The C-ABI library builds, loads and exports every function include/pi.h
declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

from paper_2406_16091_gb300 import build as pibuild
from paper_2406_16091_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(pi_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pi_create", "pi_bin", "pi_interact", "pi_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    pibuild.build()
    lib = ctypes.CDLL(pibuild.LIB)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    names = declared_functions()
    assert all(hasattr(binding, n) or n in ("pi_status_str", "pi_last_error") for n in names)
    assert binding.status_str(binding.PI_ERR_TIMEOUT) == "device-side wait timed out"
    assert binding.status_str(0) == "ok"


def test_host_side_argument_checks():
    """Argument errors are caught on the host before anything touches a GPU."""
    L = binding.load()
    out = ctypes.c_void_p()
    bad = binding.PiBox((ctypes.c_float * 3)(0, 0, 0), (ctypes.c_float * 3)(1, 0, 1))
    assert L.pi_create(ctypes.byref(bad), 0.1, 10, ctypes.byref(out)) == binding.PI_ERR_INVALID_ARG
    good = binding.PiBox((ctypes.c_float * 3)(0, 0, 0), (ctypes.c_float * 3)(1, 1, 1))
    assert L.pi_create(ctypes.byref(good), 0.0, 10, ctypes.byref(out)) == binding.PI_ERR_INVALID_ARG
    assert L.pi_create(ctypes.byref(good), float("nan"), 10, ctypes.byref(out)) == binding.PI_ERR_INVALID_ARG
    assert L.pi_create(ctypes.byref(good), 0.1, -1, ctypes.byref(out)) == binding.PI_ERR_INVALID_ARG
    # 2^31 cells is beyond the index range
    assert L.pi_create(ctypes.byref(good), 1.0 / 1291, 10, ctypes.byref(out)) == binding.PI_ERR_INVALID_ARG
    assert L.pi_bin(None, None, None, None, 0, None) == binding.PI_ERR_INVALID_ARG
    assert L.pi_interact(None, 1.0, None, None, None, None, None, 0, None) == binding.PI_ERR_INVALID_ARG
    assert L.pi_destroy(None) == binding.PI_OK


def test_destroyed_handles_are_refused_before_the_library_sees_them():
    """A context or server handle passes as its pointer until it is
    destroyed; afterwards the binding refuses it, so no call hands freed
    memory to the library (checked against a host C function)."""
    libc = ctypes.CDLL(None)
    libc.strlen.argtypes = [ctypes.c_void_p]
    libc.strlen.restype = ctypes.c_size_t
    buf = ctypes.create_string_buffer(b"seven!!")
    h = binding.Handle(ctypes.addressof(buf), "context")
    assert libc.strlen(h) == 7
    h._close()
    try:
        libc.strlen(h)
    except ctypes.ArgumentError as e:
        assert "destroyed" in str(e)
    else:
        raise AssertionError("a destroyed handle was passed on")
