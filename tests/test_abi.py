"""The C-ABI library loads and exports every symbol include/sgp.h declares
(no GPU needed: only argument validation that returns before any CUDA work)."""
import ctypes
import os
import re

import pytest

from paper_2603_25282_gb300 import sgp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "sgp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sgp_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(sgp.LIB_PATH):
        from paper_2603_25282_gb300 import build
        build.build()
    return sgp.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name


def test_version_and_status_strings(lib):
    assert lib.sgp_version() >= 100
    assert lib.sgp_status_string(0) == b"SGP_OK"
    assert lib.sgp_status_string(1) == b"SGP_EINVAL"
    assert lib.sgp_status_string(8) == b"SGP_EDRIFT"


def test_create_grid_rejects_bad_arguments_before_cuda(lib):
    with pytest.raises(sgp.SgpError, match="EINVAL"):
        sgp.create_grid((64, 64, 64, 64), 8.0)        # dim 4
    with pytest.raises(sgp.SgpError, match="EINVAL"):
        sgp.create_grid((100, 64), 8.0)               # unsupported N
    with pytest.raises(sgp.SgpError, match="EINVAL"):
        sgp.create_grid((64, 64), -1.0)               # L <= 0
    with pytest.raises(sgp.SgpError, match="EINVAL"):
        sgp.create_grid((64, 64), 8.0, batch=0)
    with pytest.raises(sgp.SgpError, match="EINVAL"):
        sgp.create_grid((64, 64), 8.0, prec=16)


def test_null_context_calls_are_rejected(lib):
    assert lib.sgp_step(None, 1, 0.1, 0) == 1
    assert lib.sgp_observables(None, None) == 1
    assert lib.sgp_record(None, 10, 0.1, 0, 0) == 1
    assert lib.sgp_set_health_check(None, 10, 1e-6) == 1
    assert lib.sgp_step_host(None, None, 0.0, None, 1, 0.1, 0, 1) == 1
    assert lib.sgp_ensemble_step_host(None, None, 0.0, None, 1, 0.1, 0) == 1
    # allocator and free function come together
    assert lib.sgp_set_allocator(sgp.ALLOC_FN(lambda *a: None), sgp.FREE_FN(), None) == 1
    assert lib.sgp_set_allocator(sgp.ALLOC_FN(), sgp.FREE_FN(), None) == 0
    assert lib.sgp_backward(None, None, 0, None, 0, None) == 1
    assert lib.sgp_destroy(None) == 0


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without libsgp.so every entry point of the binding raises."""
    monkeypatch.setattr(sgp, "_lib", None)
    monkeypatch.setattr(sgp, "LIB_PATH", str(tmp_path / "libsgp.so"))
    with pytest.raises(RuntimeError, match="not built"):
        sgp.lib()
    with pytest.raises(RuntimeError, match="not built"):
        sgp.Context((32, 32), 4.0)
    with pytest.raises(RuntimeError, match="not built"):
        sgp.substep_plan("ts2", 1, 1e-3)


def test_every_declaration_states_its_error_behaviour():
    """Each entry point of include/sgp.h is documented with its errors (or
    that it cannot fail); declarations written together share a comment."""
    txt = open(os.path.join(ROOT, "include", "sgp.h")).read()
    decl = re.compile(r"(?:sgp_status|int|long long|const char\*|void)\s+\**(sgp_[a-z_]+)\s*\([^;]*\);", re.S)
    words = ("Error", "SGP_E", "Cannot fail", "for NULL", "no-op", "Always SGP_OK", "alid until")
    missing = []
    for m in decl.finditer(txt):
        head = txt[:m.start()]
        end = head.rfind("*/")
        start = head.rfind("/*", 0, end)
        between = head[end + 2:]
        # only other declarations may sit between the comment and this one
        if end < 0 or decl.sub("", between).strip():
            missing.append(m.group(1))
            continue
        if not any(w in head[start:end] for w in words):
            missing.append(m.group(1))
    assert not missing, missing
