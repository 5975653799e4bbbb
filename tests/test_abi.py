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


def test_struct_layouts_match_header(tmp_path):
    """The binding's ctypes structures have the C layout of include/bsm.h
    (sizes and field offsets, printed by a C program compiled against it)."""
    import ctypes

    from paper_1705_10218_gb300 import bsm

    structs = {"bsm_opts": bsm._Opts, "bsm_stats": bsm._Stats, "bsm_profile": bsm._Profile}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bsm.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines():
        cname, f, v = ln.split()
        got[(cname, f)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_fp64_kernel_numbers_match_header():
    src = open(os.path.join(ROOT, "include", "bsm.h")).read()
    nums = {m.group(1): int(m.group(2)) for m in re.finditer(r"(BSM_FP64_\w+)\s*=\s*(\d+)", src)}
    from paper_1705_10218_gb300 import bsm

    assert nums and all(getattr(bsm, k) == v for k, v in nums.items())
