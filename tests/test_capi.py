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


# ------------------------------------------------------------ struct layouts
_STRUCTS = ["hse_params", "hse_eval_stats", "hse_server_config", "hse_request", "hse_server_stats",
            "hse_instance", "hse_batch_stats", "hse_pipe_peaks"]


def _header_fields(text, name):
    """Field names of `typedef struct { ... } name;` in declaration order."""
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", text).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(","):
            m = re.search(r"([A-Za-z_]\w*)\s*(\[[^\]]*\])?\s*$", part.strip())
            fields.append(m.group(1))
    return fields


def test_binding_structs_mirror_the_header():
    """Each ctypes structure of the binding has the header's fields in the same
    order, and gcc's sizeof / offsetof of the header's structs equal ctypes'
    (a field added on one side only would shift every later field)."""
    import shutil
    import subprocess
    import tempfile
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "hse.h")).read(), flags=re.S)
    lines = ['#include <stdio.h>', '#include "hse.h"', "int main(void) {"]
    for s in _STRUCTS:
        names = _header_fields(text, s)
        py = getattr(hse, s)
        assert [f[0] for f in py._fields_] == names, s
        lines.append(f'  printf("{s} %zu\\n", sizeof({s}));')
        for f in names:
            lines.append(f'  printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("  return 0;\n}")
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(line.split() for line in out if line.strip())
    for s in _STRUCTS:
        py = getattr(hse, s)
        assert int(got[s]) == ctypes.sizeof(py), s
        for f in [f[0] for f in py._fields_]:
            assert int(got[f"{s}.{f}"]) == getattr(py, f).offset, f"{s}.{f}"


def test_binding_constants_match_the_header():
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "hse.h")).read(), flags=re.S)
    for name, value in re.findall(r"\b(HSE_[A-Z0-9_]+)\s*=\s*(\d+)", text):
        if hasattr(hse, name):
            assert getattr(hse, name) == int(value), name
    for name in ("HSE_FFT_AUTO", "HSE_FFT_CUFFT", "HSE_FFT_DF64", "HSE_FP64", "HSE_MIXED", "HSE_FREE_SPACE"):
        assert hasattr(hse, name), name
