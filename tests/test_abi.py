"""The C-ABI library: it builds, loads, exports every symbol include/ppf.h
declares, and its host-side argument checks and fault injection work without
a GPU (no compute call is made here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    hdr = open(os.path.join(ROOT, "include", "ppf.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(ppf_[a-z0-9_]+)\s*\(", hdr)))


@pytest.fixture(scope="module")
def lib():
    import paper_1310_5045_gb300 as p
    return p.load()


def test_exports_every_declared_symbol(lib):
    names = declared()
    assert "ppf_create" in names and "ppf_resample" in names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    import paper_1310_5045_gb300 as p
    for s in range(7):
        assert p.status_string(s).startswith("PPF_")
    assert p.status_string(99) == "PPF_UNKNOWN"


def _model(**kw):
    import paper_1310_5045_gb300 as p
    m = p.Model(**kw)
    return m.c()


@pytest.mark.parametrize("kw,n,gs", [
    ({}, 0, 1), ({}, 10, 0), ({}, 10, 11), ({"patch_radius": 9}, 10, 1), ({"patch_radius": -1}, 10, 1),
    ({"psf_sigma": 0.0}, 10, 1), ({"sigma_xi": -1.0}, 10, 1), ({"width": 0}, 10, 1),
    ({"frame_dtype": 7}, 10, 1), ({"sigma_m": float("nan")}, 10, 1), ({}, 2**31, 1),
])
def test_create_rejects_invalid_arguments(lib, kw, n, gs):
    ctx = C.c_void_p()
    assert lib.ppf_create(C.byref(_model(**kw)), n, gs, None, C.byref(ctx)) == 1  # PPF_EINVAL
    assert not ctx


def test_null_arguments(lib):
    assert lib.ppf_step(None, None, 1) == 1
    assert lib.ppf_resample(None, 0, 0.0) == 1
    assert lib.ppf_estimate(None, None) == 1
    assert lib.ppf_set_particles(None, None, None, None) == 1
    lib.ppf_destroy(None)
    assert lib.ppf_last_error(None) == b""


def test_injected_allocation_failure(lib, monkeypatch):
    monkeypatch.setenv("PPF_FAULT", "alloc")
    ctx = C.c_void_p()
    assert lib.ppf_create(C.byref(_model()), 100, 10, None, C.byref(ctx)) == 2  # PPF_ENOMEM
    assert not ctx


def test_no_device_is_reported_not_crashed(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    ctx = C.c_void_p()
    st = lib.ppf_create(C.byref(_model()), 100, 10, None, C.byref(ctx))
    assert st in (2, 3)  # ENOMEM / ECUDA, never a crash
    assert not ctx
