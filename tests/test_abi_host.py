"""Host-side checks of the C-ABI library (no GPU compute calls)."""
import os
import re

import pytest

from paper_1908_11246_gb300 import build, vup

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return vup.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "vup.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vup_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    fns = declared_functions()
    for name in ["vup_grid_create", "vup_eval_model", "vup_propagate", "vup_ipsa_sensitivity"]:
        assert name in fns


def test_library_exports_every_declared_symbol(L):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", vup.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (vup_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    for f in declared_functions():
        assert hasattr(L, f)


def test_binding_names_match_header():
    assert sorted(vup.ABI_SYMBOLS) == declared_functions()


def test_status_strings(L):
    for code in range(9):
        assert vup.vup_status_string(code).startswith("VUP_")
    assert vup.vup_status_string(vup.VUP_ERR_BOUNDS).startswith("VUP_ERR_BOUNDS")
    assert "sm_103a" in vup.vup_version()


def test_grid_create_rejects_bad_shapes_on_host(L):
    import ctypes as C
    h = C.c_void_p()
    n = (C.c_int64 * 3)(10, 10, 10)
    lo = (C.c_double * 3)(0, 0, 0)
    hi = (C.c_double * 3)(1, 1, 1)
    assert L.vup_grid_create(0, n, lo, hi, C.byref(h)) == vup.VUP_ERR_INVALID_ARG
    assert L.vup_grid_create(4, n, lo, hi, C.byref(h)) == vup.VUP_ERR_INVALID_ARG
    bad_n = (C.c_int64 * 1)(0)
    assert L.vup_grid_create(1, bad_n, lo, hi, C.byref(h)) == vup.VUP_ERR_INVALID_ARG
    big_n = (C.c_int64 * 1)(40000)
    assert L.vup_grid_create(1, big_n, lo, hi, C.byref(h)) == vup.VUP_ERR_INVALID_ARG
    inv = (C.c_double * 1)(2.0)
    assert L.vup_grid_create(1, n, inv, hi, C.byref(h)) == vup.VUP_ERR_INVALID_ARG
    nan = (C.c_double * 1)(float("nan"))
    assert L.vup_grid_create(1, n, nan, hi, C.byref(h)) == vup.VUP_ERR_INVALID_ARG
    assert L.vup_grid_create(1, n, lo, hi, None) == vup.VUP_ERR_INVALID_ARG


def test_calls_reject_null_grid_on_host(L):
    d = vup.vup_densities()
    assert L.vup_propagate(None, None, 1, None, None, None, None) == vup.VUP_ERR_INVALID_ARG
    assert L.vup_eval_model(None, 2, None, 0, 16, 4, None) == vup.VUP_ERR_INVALID_ARG
    assert L.vup_ipsa_sensitivity(None, None, 1, None, None, None, None) == vup.VUP_ERR_INVALID_ARG
    assert L.vup_propagate_weights(None, 1, None, None, None, None) == vup.VUP_ERR_INVALID_ARG
    assert L.vup_grid_destroy(None) == vup.VUP_ERR_INVALID_ARG
    assert L.vup_sync(None, None) == vup.VUP_ERR_INVALID_ARG


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(vup, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(vup, "_lib", None)
    with pytest.raises(ImportError):
        vup.lib()


def test_allocation_failure_hook_on_host(L):
    """With the hook armed, grid creation fails with VUP_ERR_OOM at its first
    device allocation (no CUDA device is needed to reach it) and returns no
    handle; the detail names the failing allocation."""
    import ctypes as C
    h = C.c_void_p(1234)
    n = (C.c_int64 * 2)(10, 10)
    lo = (C.c_double * 2)(0, 0)
    hi = (C.c_double * 2)(1, 1)
    vup.vup_debug_fail_alloc(0)
    try:
        assert L.vup_grid_create(2, n, lo, hi, C.byref(h)) == vup.VUP_ERR_OOM
        assert not h.value
        assert "cudaErrorMemoryAllocation" in vup.vup_last_error_detail()
    finally:
        vup.vup_debug_fail_alloc(-1)


C_PROGRAM = r"""
#include "vup.h"
#include <stdio.h>
#include <string.h>

/* A C99 caller of the boundary: the header alone, linked against libvup.so;
   only calls that need no device. */
int main(void) {
    int fails = 0;
    vup_grid g = NULL;
    const int64_t n[2] = {10, 10};
    const double lo[2] = {0.0, 0.0}, hi[2] = {1.0, 1.0};
    vup_densities d;
    int s;
    memset(&d, 0, sizeof d);
    if (strstr(vup_version(), "sm_103a") == NULL) ++fails;
    for (s = 0; s <= VUP_ERR_BOUNDS; ++s)
        if (strncmp(vup_status_string((vup_status)s), "VUP_", 4) != 0) ++fails;
    if (vup_grid_create(0, n, lo, hi, &g) != VUP_ERR_INVALID_ARG || g != NULL) ++fails;
    if (vup_propagate(NULL, &d, VUP_BF16X3, NULL, NULL, NULL, NULL) != VUP_ERR_INVALID_ARG) ++fails;
    if (vup_propagate_weights(NULL, 0, NULL, NULL, NULL, NULL) != VUP_ERR_INVALID_ARG) ++fails;
    if (vup_set_weights_form(NULL, 0) != VUP_ERR_INVALID_ARG) ++fails;
    if (vup_set_hist_stream(NULL, 0, NULL) != VUP_ERR_INVALID_ARG) ++fails;
    if (vup_sync(NULL, NULL) != VUP_ERR_INVALID_ARG) ++fails;
    printf("%s %d\n", fails ? "FAIL" : "OK", fails);
    return fails != 0;
}
"""


def test_header_compiles_as_c99_and_links(L, tmp_path):
    """include/vup.h compiles as strict C99 without warnings and a C program
    links against libvup.so and calls it (host-only calls)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "caller.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "caller"
    libdir = os.path.dirname(vup.LIB_PATH)
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           str(src), "-o", str(exe), "-L", libdir, "-l:" + os.path.basename(vup.LIB_PATH), "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr
