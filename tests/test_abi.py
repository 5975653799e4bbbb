"""The C ABI without a GPU: libbsm builds for sm_103a, loads, and exports every
function declared in include/*.h; the binding's error codes match the header."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(bsm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("bsm_ctx_create", "bsm_mat_create", "bsm_multiply", "bsm_mat_get_values"):
        assert must in names


def test_library_builds_and_exports(bsm_lib):
    lib = bsm_lib.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", bsm_lib.lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_error_codes_match_header(bsm_lib):
    src = open(os.path.join(ROOT, "include", "bsm.h")).read()
    codes = {m.group(1): int(m.group(2)) for m in re.finditer(r"BSM_ERR_(\w+)\s*=\s*(-?\d+)", src)}
    from paper_1705_10218_gb300 import bsm

    for name, code in codes.items():
        assert bsm.ERRORS[code] == name
    assert bsm_lib.lib().bsm_strerror(-5) == b"C aliases A or B"


def test_no_cpu_fallback_without_library(tmp_path, monkeypatch):
    """The binding raises when libbsm.so is missing instead of computing anything."""
    from paper_1705_10218_gb300 import bsm

    monkeypatch.setattr(bsm, "lib_path", str(tmp_path / "missing.so"))
    monkeypatch.setattr(bsm, "_lib", None)
    with pytest.raises(RuntimeError):
        bsm.Context(0)
