"""C ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every entry point that include/dect.h declares; argument checks run
on the host before any CUDA call."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dect.h")

nvcc_missing = shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dect_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if nvcc_missing:
        pytest.skip("no CUDA toolkit to build libdect")
    from paper_1607_01650_gb300 import _build
    path = _build.build()
    return C.CDLL(path), path


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dect_plan_create", "dect_plan_destroy", "dect_project", "dect_backproject",
                     "dect_adm_tv", "dect_pls_decompose", "dect_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    cdll, path = lib
    missing = [n for n in declared_functions() if not hasattr(cdll, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dect_[a-z0-9_]+)", out))
    assert set(declared_functions()) <= exported


def test_binding_covers_the_header(lib):
    import paper_1607_01650_gb300 as dect
    assert set(declared_functions()) <= set(dect._SIGS)


def test_built_for_sm_103a_only():
    from paper_1607_01650_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_side_argument_checks(lib):
    import paper_1607_01650_gb300 as dect
    L = dect.load()
    assert L.dect_status_string(0) == b"ok"
    assert L.dect_status_string(1) == b"invalid argument"
    assert L.dect_version() >= 100
    # NULL plan / pointers and bad geometry are refused before any CUDA call
    assert L.dect_project(None, None, None, 1, None) == 1
    assert L.dect_backproject(None, None, None, 1, None) == 1
    assert L.dect_pls_decompose(None, 4, 1, None, None, None, None) == 1
    out = C.c_void_p()
    bad = dect._Geometry(0, 1.0, 10, 10, 1.0, 100.0, 200.0, 0.0, 6.28, 0.0)   # n = 0
    assert L.dect_plan_create(C.byref(bad), 0, None, C.byref(out)) == 1
    bad = dect._Geometry(64, 1.0, 10, 10, 1.0, 20.0, 200.0, 0.0, 6.28, 0.0)   # source inside the image
    assert L.dect_plan_create(C.byref(bad), 0, None, C.byref(out)) == 1
    bad = dect._Geometry(64, 1.0, 10, 10, 1.0, 100.0, 50.0, 0.0, 6.28, 0.0)   # SDD < SOD
    assert L.dect_plan_create(C.byref(bad), 0, None, C.byref(out)) == 1
    assert L.dect_plan_destroy(None) == 0
    assert L.dect_plan_get_tuning(None, 2, None, None) == 1
    assert L.dect_plan_get_tv_tuning(None, 2, None, None) == 1
    assert L.dect_plan_set_tv_tuning(None, 2, 0) == 1
    prm = dect.AdmParams()._c()
    grp = (dect._AdmGroup * 1)()
    assert L.dect_adm_tv_batch_ex(None, 1, C.byref(prm), dect.PROJ_TABLE, None) == 1  # no groups
    assert L.dect_adm_tv_batch_ex(grp, 0, C.byref(prm), 2, None) == 1                 # unknown projector
    assert L.dect_adm_tv_batch_ex(grp, 0, C.byref(prm), dect.PROJ_TABLE, None) == 0   # nothing to do
    assert L.dect_cnn_set_conv_path(None, 0) == 1
    assert L.dect_cnn_get_conv_path(None) == -1
    assert L.dect_cnn_check(None) == 1


def test_struct_layouts_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the field offsets and size
    that a C compiler gives the struct of the same name in include/dect.h."""
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    import paper_1607_01650_gb300 as dect
    pairs = {"dect_geometry": dect._Geometry, "dect_plan_info": dect._PlanInfo,
             "dect_adm_params": dect._AdmParams, "dect_adm_report": dect._AdmReport,
             "dect_adm_profile": dect._AdmProfile, "dect_adm_group": dect._AdmGroup,
             "dect_pls_params": dect._PlsParams, "dect_pls_report": dect._PlsReport}
    lines = ["#include <stdio.h>", '#include "dect.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in pairs.items():
        assert got[(cname, "sizeof")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_variant_count_matches_the_header():
    import paper_1607_01650_gb300 as dect
    m = re.search(r"#define\s+DECT_BWD_VARIANTS\s+(\d+)", open(HEADER).read())
    assert m and int(m.group(1)) == dect.BWD_VARIANTS
    m = re.search(r"#define\s+DECT_FWD_VARIANTS\s+(\d+)", open(HEADER).read())
    assert m and int(m.group(1)) == dect.FWD_VARIANTS
    m = re.search(r"#define\s+DECT_TV_VARIANTS\s+(\d+)", open(HEADER).read())
    assert m and int(m.group(1)) == dect.TV_VARIANTS


def test_checked_library_exports_and_host_checks(lib):
    """The checked build exports every entry point; the plain build refuses an
    out-of-range self-test index on the host (its kernel has no check)."""
    from paper_1607_01650_gb300 import _build
    chk = C.CDLL(_build.LIB_CHECKED)
    missing = [n for n in declared_functions() if not hasattr(chk, n)]
    assert not missing, missing
    assert chk.dect_checked_build() == 1
    cdll, _ = lib
    assert cdll.dect_checked_build() == 0
    cdll.dect_selftest_index.argtypes = [C.c_int, C.c_void_p]
    assert cdll.dect_selftest_index(8, None) == 1   # DECT_ERR_INVALID_ARG, nothing enqueued
    assert cdll.dect_selftest_index(-1, None) == 1
