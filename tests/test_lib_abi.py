"""The CUDA library builds, loads without a GPU, and exports every entry
point include/pbng.h declares (no compute calls here)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pbng_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2306_09021_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared("pbng.h")
    for n in ("pbng_create_mesh", "pbng_set_constraints", "pbng_sweep", "pbng_solve",
              "pbng_get_colouring", "pbng_residual", "pbng_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for header in os.listdir(os.path.join(ROOT, "include")):
        for name in _declared(header):
            assert hasattr(lib, name), f"{name} declared in {header} but not exported"


def test_binding_signatures_cover_the_header(lib):
    from paper_2306_09021_gb300 import _lib
    assert set(_lib.SIGNATURES) == set(_declared("pbng.h"))


def test_params_struct_layout(lib):
    from paper_2306_09021_gb300 import _lib
    p = _lib.PbngParams()
    lib.pbng_default_params.argtypes = [ctypes.POINTER(_lib.PbngParams)]
    lib.pbng_default_params(ctypes.byref(p))  # host-only: fills defaults
    assert (p.omega, p.rho, p.gamma, p.step, p.residual_every) == (1.7, 0.95, 1.7, 1.0, 10)
    assert p.precision == 1 and p.accel == 0 and p.resume == 0


def test_status_strings(lib):
    lib.pbng_status_string.restype = ctypes.c_char_p
    assert lib.pbng_status_string(0) == b"ok"
    assert lib.pbng_status_string(7) == b"not converged"


def _header_constants():
    """Every `NAME = value` enumerator and `#define NAME value` of pbng.h."""
    text = open(os.path.join(ROOT, "include", "pbng.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    consts = {k: int(v) for k, v in re.findall(r"\b(PBNG_[A-Z_0-9]+)\s*=\s*(-?\d+)", text)}
    consts.update({k: int(v) for k, v in re.findall(r"#define\s+(PBNG_[A-Z_0-9]+)\s+(\d+)", text)})
    return consts


def test_binding_constants_match_the_header():
    """The binding's names for the accelerations, precisions, models and
    colour orders, and its size limits, are the header's values."""
    from paper_2306_09021_gb300 import _lib
    c = _header_constants()
    maps = [(_lib.ACCEL, "PBNG_ACCEL_"), (_lib.PRECISION, "PBNG_PREC_"), (_lib.MODEL, "PBNG_MODEL_"),
            (_lib.ORDER, "PBNG_ORDER_")]
    for table, prefix in maps:
        declared = {k[len(prefix):].lower(): v for k, v in c.items() if k.startswith(prefix)}
        assert table == declared, prefix
    assert _lib.MAX_COLOURS == c["PBNG_MAX_COLOURS"]
    assert _lib.MAX_CTAS_PER_SM == c["PBNG_MAX_CTAS_PER_SM"]
    assert _lib.MAX_SOLVE_EVENTS == c["PBNG_MAX_SOLVE_EVENTS"]
