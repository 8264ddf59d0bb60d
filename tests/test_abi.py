"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry point
that include/jaxshock.h declares.  CPU only: no compute calls."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "jaxshock.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(js_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("js_create", "js_rhs", "js_step", "js_rhs_vjp", "js_step_vjp", "js_max_dt", "js_destroy",
                     "js_sync_status", "js_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2601_04400_gb300 import build
    try:
        path = build.build()
    except (OSError, RuntimeError) as e:  # pragma: no cover - nvcc missing
        pytest.skip("nvcc unavailable: %s" % e)
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2601_04400_gb300 import binding
    assert set(_declared()) <= set(binding.SIGNATURES), set(_declared()) - set(binding.SIGNATURES)


def test_strerror_needs_no_gpu():
    from paper_2601_04400_gb300 import binding
    assert binding.strerror(0) == "ok"
    assert "non-physical" in binding.strerror(-3)
