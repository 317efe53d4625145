"""The C-ABI library builds, loads without a GPU and exports every symbol pavg.h declares."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "pavg.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(pavg_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2103_07706_gb300 import build
    return build.build()


def test_header_declares_the_api():
    syms = declared_symbols()
    for name in ("pavg_create", "pavg_expL_apply", "pavg_averaged_rhs", "pavg_timestep", "pavg_nonlinear"):
        assert name in syms


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_names_match_header(libpath):
    from paper_2103_07706_gb300 import pavg
    assert sorted(pavg.EXPORTED) == declared_symbols()


def test_binding_constants_match_header():
    """Every numeric #define of the header that the binding names has the
    same value there (error codes, modes, the exponential width limit)."""
    from paper_2103_07706_gb300 import pavg
    text = open(os.path.join(ROOT, "include", "pavg.h")).read()
    defs = dict(re.findall(r"#define\s+(PAVG_\w+)\s+\(?(-?[0-9.]+)\)?", text))
    assert "PAVG_MAX_CHEB_ARG" in defs and "PAVG_ERR_INVAL" in defs
    named = {k: v for k, v in defs.items() if hasattr(pavg, k)}
    assert "PAVG_MAX_CHEB_ARG" in named
    for k, v in named.items():
        assert float(getattr(pavg, k)) == float(v), k


def test_default_params_and_invalid_create_without_gpu(libpath):
    """Host-only calls: defaults, argument checks (no device work happens)."""
    from paper_2103_07706_gb300 import pavg
    p = pavg.default_params()
    assert p.refinement == 3 and p.cheb_tol == 1e-6 and p.g == 9.80616 and p.H == 5000.0
    lib = pavg.lib()
    h = ctypes.c_void_p()
    bad = pavg.default_params(refinement=-1)
    assert lib.pavg_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad = pavg.default_params(cheb_tol=0.0)
    assert lib.pavg_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad = pavg.default_params(quad_rule=7)
    assert lib.pavg_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    assert lib.pavg_destroy(None) == -1
    assert lib.pavg_averaged_rhs(None, 1.0, 4, None, None, None) == -1
    assert lib.pavg_last_error(None) == b"null context"


def test_batch_and_surrogate_argument_checks_without_gpu(libpath):
    from paper_2103_07706_gb300 import pavg
    lib = pavg.lib()
    h = ctypes.c_void_p()
    assert lib.pavg_batch_create(None, 0, ctypes.byref(h)) == -1
    assert lib.pavg_batch_create(None, 2, ctypes.byref(h)) == -1
    assert lib.pavg_batch_destroy(None) == -1
    assert lib.pavg_batch_averaged_rhs(None, None, None, None, None, None) == -1
    assert lib.pavg_batch_timestep(None, None, None, None, None, 1, None) == -1
    assert lib.pavg_batch_set_config(None, None) == -1
    assert lib.pavg_batch_last_error(None) == b"null batch"
    assert lib.pavg_surrogate_create(0, 1, ctypes.byref(h)) == -1
    assert lib.pavg_surrogate_create(5000, 1, ctypes.byref(h)) == -1
    assert lib.pavg_surrogate_destroy(None) == -1
    assert lib.pavg_surrogate_train(None, 1, 16, 1e-3, 1, None, None) == -1
    assert lib.pavg_surrogate_last_error(None) == b"null surrogate"
