"""The C-ABI library builds for sm_103a, loads, exports every entry point that
include/irs.h declares, and agrees with the ctypes binding on struct layout.
Host-only checks: no kernel runs here."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2204_10871_gb300 import build as libbuild
from paper_2204_10871_gb300 import irs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "irs.h")


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return C.CDLL(libbuild.LIB)


def declared_entry_points():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(irs_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for want in ("irs_plan", "irs_plan_info_get", "irs_make_map", "irs_make_maps_batched",
                 "irs_shoot_rays", "irs_plan_sync", "irs_plan_destroy", "irs_status_str"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_entry_points():
        assert hasattr(lib, name), f"{name} declared in irs.h but not exported"


def test_exports_have_c_linkage():
    out = subprocess.run(["nm", "-D", "--defined-only", libbuild.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (irs_[a-z_0-9]+)$", out, flags=re.M))
    assert set(declared_entry_points()) <= exported


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "irs.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("irs_params %zu\n", sizeof(irs_params));
  printf("irs_plan_info %zu\n", sizeof(irs_plan_info));
  P(irs_params, n_star) P(irs_params, method) P(irs_params, cell_mult) P(irs_params, kernel_variant)
  P(irs_params, reserved)
  P(irs_plan_info, n_rays) P(irs_plan_info, ncell_x) P(irs_plan_info, workspace_bytes)
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(line.rsplit(" ", 1) for line in subprocess.check_output([str(exe)], text=True)
               .strip().splitlines())
    assert int(got["irs_params"]) == C.sizeof(irs.IrsParams)
    assert int(got["irs_plan_info"]) == C.sizeof(irs.IrsPlanInfo)
    for key, val in got.items():
        if "." in key:
            struct, field = key.split(".")
            cls = irs.IrsParams if struct == "irs_params" else irs.IrsPlanInfo
            assert int(val) == getattr(cls, field).offset, key


def test_status_strings(lib):
    lib.irs_status_str.restype = C.c_char_p
    for code in range(9):
        assert lib.irs_status_str(code)
    assert b"degenerate" in lib.irs_status_str(2)


def test_host_validation_without_device(lib):
    """Argument checks and the degenerate-map check happen on the host before
    any CUDA call, so they answer without a GPU."""
    h = C.c_void_p()
    lib.irs_plan.argtypes = [C.POINTER(irs.IrsParams), C.c_void_p, C.POINTER(C.c_void_p)]
    good = irs.make_params(0.3, 0.0, 0.3, (-2.5, 2.5, -2.5, 2.5), 128, 25.0)
    bad_pix = irs.make_params(0.3, 0.0, 0.3, (-2.5, 2.5, -2.5, 2.5), 0, 25.0)
    assert lib.irs_plan(C.byref(bad_pix), None, C.byref(h)) == 1
    bad_src = irs.make_params(0.3, 0.0, 0.3, (2.5, -2.5, -2.5, 2.5), 128, 25.0)
    assert lib.irs_plan(C.byref(bad_src), None, C.byref(h)) == 1
    nan = irs.make_params(float("nan"), 0.0, 0.3, (-2.5, 2.5, -2.5, 2.5), 128, 25.0)
    assert lib.irs_plan(C.byref(nan), None, C.byref(h)) == 1
    degenerate = irs.make_params(0.5, 0.0, 0.5, (-1, 1, -1, 1), 16, 4.0)
    assert lib.irs_plan(C.byref(degenerate), None, C.byref(h)) == 2
    flags = irs.make_params(0.3, 0.0, 0.3, (-2.5, 2.5, -2.5, 2.5), 128, 25.0)
    flags.flags = 1
    assert lib.irs_plan(C.byref(flags), None, C.byref(h)) == 1
    assert lib.irs_plan(None, None, C.byref(h)) == 1
    assert lib.irs_plan(C.byref(good), None, None) == 1
    lib.irs_plan_destroy.argtypes = [C.c_void_p]
    assert lib.irs_plan_destroy(None) == 0
    lib.irs_make_map.argtypes = [C.c_void_p] * 3 + [C.c_int64] + [C.c_void_p] * 3
    assert lib.irs_make_map(None, None, None, 0, None, None, None) == 1
