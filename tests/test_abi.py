"""CPU-only checks of the C-ABI boundary: the library builds for sm_103a,
loads, and exports every entry point that include/sw.h declares, with the
binding's table in the same set.  No compute call needs a GPU here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "sw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sw_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libsw():
    from paper_2607_00117_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_four_calls():
    syms = declared_symbols()
    for s in ("sw_set_potential", "sw_integrate_library", "sw_project", "sw_solve_weights"):
        assert s in syms


def test_every_declared_symbol_is_exported(libsw):
    missing = [s for s in declared_symbols() if not hasattr(libsw, s)]
    assert not missing, missing


def test_binding_matches_header():
    from paper_2607_00117_gb300 import sw
    assert sorted(sw.SIGNATURES) == declared_symbols()


def test_no_internal_symbols_exported(libsw):
    # internal C++ entry points stay hidden (visibility=hidden build)
    for name in ("_ZN2sw6gram_tcEP6sw_ctxPK13__nv_bfloat16llPfPi",):
        assert not hasattr(libsw, name)


def test_create_without_gpu_fails_cleanly(libsw):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2607_00117_gb300 import sw
    with pytest.raises(sw.SwError):
        sw.Context(0, "fp32")
