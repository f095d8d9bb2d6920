"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/sme.h declares.
Host-side argument and CSR validation returns its status codes before any device work,
so those paths are checked here without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1602_06621_gb300 import sme

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(sme_\w+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = sme.load()
    names = _declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
        assert name in sme.SIGNATURES, f"binding lacks {name}"


def test_status_strings():
    assert sme.sme_status_string(0) == "ok"
    assert sme.sme_status_string(-2) == "invalid CSR"


def _csr():
    rp = np.array([0, 2, 3, 5], np.int32)
    col = np.array([0, 2, 1, 0, 3], np.int32)
    val = np.array([1.0, -2.0, 3.0, 0.5, 4.0])
    return rp, col, val


@pytest.mark.parametrize("mutate,code", [
    (lambda rp, col, val: rp.__setitem__(1, 4), "SME_ERR_INVALID_CSR"),        # row_ptr decreases
    (lambda rp, col, val: col.__setitem__(4, 9), "SME_ERR_INVALID_CSR"),       # column out of range
    (lambda rp, col, val: col.__setitem__(1, 0), "SME_ERR_INVALID_CSR"),       # repeated column
    (lambda rp, col, val: rp.__setitem__(3, 4), "SME_ERR_INVALID_CSR"),        # row_ptr[m] != nnz
    (lambda rp, col, val: val.__setitem__(2, np.nan), "SME_ERR_NONFINITE"),    # NaN value
    (lambda rp, col, val: val.__setitem__(0, np.inf), "SME_ERR_NONFINITE"),    # Inf value
])
def test_host_csr_validation(mutate, code):
    rp, col, val = _csr()
    mutate(rp, col, val)
    with pytest.raises(sme.SmeError) as ei:
        sme.sme_op_create_csr(3, 4, rp, col, val, stream=0)
    assert ei.value.name == code


def test_degenerate_shapes_are_rejected():
    rp, col, val = _csr()
    with pytest.raises(sme.SmeError) as ei:
        sme.sme_op_create_csr(0, 4, np.zeros(1, np.int32), col[:0], val[:0], stream=0)
    assert ei.value.name == "SME_ERR_ARG"
    lib = sme.load()
    p = sme.sme_equil_params(0, 0, 0, 0, 10, 32, 1, 0, 0, 0, 0)
    assert lib.sme_equilibrate(None, ctypes.byref(p), None, None, None, None, None) == -1


def _prototypes():
    """Parameter lists of every function include/sme.h declares, comments removed: name -> [parameter text]."""
    out = {}
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for name, params in re.findall(r"\b(sme_\w+)\s*\(([^()]*)\)\s*;", text):
            params = params.strip()
            out[name] = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
    return out


def test_binding_argument_lists_match_the_header():
    """The ctypes binding declares as many arguments as the header, pointers where the header has pointers
    and 64-bit integers where it has 64-bit integers, so a drifting signature fails here rather than
    corrupting a call."""
    protos = _prototypes()
    assert len(protos) == len(_declared())
    for name, params in protos.items():
        argtypes, _ = sme.SIGNATURES[name]
        assert len(argtypes) == len(params), (name, params)
        for p, a in zip(params, argtypes):
            is_ptr = "*" in p or p.split()[0] in ("sme_op", "sme_batch", "sme_mlp")
            if is_ptr:
                assert a is ctypes.c_void_p or issubclass(a, ctypes._Pointer) or a is ctypes.c_char_p, (name, p)
            elif p.split()[0] in ("int64_t",):
                assert a is ctypes.c_int64, (name, p)
            elif p.split()[0] in ("uint64_t",):
                assert a is ctypes.c_uint64, (name, p)
            elif p.split()[0] in ("double",):
                assert a is ctypes.c_double, (name, p)
            elif p.split()[0] in ("float",):
                assert a is ctypes.c_float, (name, p)
