"""The C ABI library builds, loads and exports every symbol include/hse.h
declares (no GPU needed); the binding carries the same names."""
import ctypes
import os
import re

import pytest

from paper_1802_07844_gb300 import build, hse

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "hse.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hse_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    path = build.build_library()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "hse_eval" in names and "hse_plan_create" in names
    for n in names:
        assert hasattr(lib, n), n
        assert hasattr(hse, n), f"binding lacks {n}"


def test_status_strings_without_gpu():
    hse.load()
    assert hse.status_name(0) == "HSE_OK"
    assert hse.status_name(1) == "HSE_ERR_INVALID"
    assert hse.status_name(6) == "HSE_ERR_UNSUPPORTED"


def test_invalid_plan_arguments_rejected_on_host():
    """Argument checks that happen before any device call."""
    with pytest.raises(hse.HseError) as e:
        hse.hse_plan_create(0, (1, 1, 1), 5.0, 0.5, 16, 1e-8)
    assert e.value.status == hse.HSE_ERR_INVALID
    with pytest.raises(hse.HseError) as e:
        hse.hse_plan_create(1, (1, -1, 1), 5.0, 0.5, 16, 1e-8)
    assert e.value.status == hse.HSE_ERR_INVALID
    with pytest.raises(hse.HseError) as e:
        hse.hse_plan_create(1, (1, 1, 1), 0.0, 0.0, 16, 0.0)
    assert e.value.status == hse.HSE_ERR_INVALID


def test_library_has_no_oracle_dependency():
    """The product library links nothing from oracle/."""
    path = build.build_library()
    data = open(path, "rb").read()
    assert b"oracle_" not in data and b"hs_oracle" not in data
