"""The C-ABI library loads without a GPU, exports what include/lse.h
declares, lays its structs out as the header does, and rejects bad
arguments before touching a device."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lse.h")


@pytest.fixture(scope="module")
def lse():
    from paper_1409_7474_gb300 import _build
    if not os.path.exists(_build.LIB):
        _build.build()
    import paper_1409_7474_gb300.lse as lse
    return lse


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lse_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lse):
    names = declared_functions()
    assert names == sorted(lse.SYMBOLS)
    lib = lse.raw_library()
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lse.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}\b", out), n


def test_struct_layout_matches_header(lse, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "lse.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(lse_params),"
        " sizeof(lse_stats), offsetof(lse_stats, c_plus), offsetof(lse_stats, norm),"
        " offsetof(lse_stats, status), offsetof(lse_params, order),"
        " offsetof(lse_params, padding));return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert vals == [ctypes.sizeof(lse.Params), ctypes.sizeof(lse.Stats),
                    lse.Stats.c_plus.offset, lse.Stats.norm.offset,
                    lse.Stats.status.offset, lse.Params.order.offset,
                    lse.Params.padding.offset]


def test_problem_layout_matches_header(lse, tmp_path):
    src = tmp_path / "problem.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "lse.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu\\n\", sizeof(lse_problem),"
        " offsetof(lse_problem, g), offsetof(lse_problem, params),"
        " offsetof(lse_problem, phi_out), offsetof(lse_problem, mask_out));return 0;}\n")
    exe = tmp_path / "problem"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert vals == [ctypes.sizeof(lse.Problem), lse.Problem.g.offset, lse.Problem.params.offset,
                    lse.Problem.phi_out.offset, lse.Problem.mask_out.offset]


def test_version_and_errors_without_gpu(lse):
    lib = lse.raw_library()
    assert lse.version() == "0.1.0"
    h = ctypes.c_void_p()
    assert lib.lse_create(None, 0, 16, 1) == lse.LSE_ERR_INVALID_ARG
    assert lib.lse_create(ctypes.byref(h), 0, 0, 1) == lse.LSE_ERR_INVALID_ARG
    assert lib.lse_create(ctypes.byref(h), 0, 16, 9) == lse.LSE_ERR_INVALID_ARG
    assert b"max_bands" in lib.lse_last_error(None)
    p = lse.Params(0, 15.0, 1.0, 9, 10, 1, 0.0, 0)
    assert lib.lse_evolve(None, None, 0, 8, 8, 1, None, None, ctypes.byref(p),
                          None, None, None, None) == lse.LSE_ERR_INVALID_ARG
    assert lib.lse_precompute_edge(None, None, 0, 8, 8, 1, 1.0, 9, 255.0,
                                   None, None) == lse.LSE_ERR_INVALID_ARG
    st = lse.Stats()
    assert lib.lse_get_stats(None, ctypes.byref(st)) == lse.LSE_ERR_INVALID_ARG
    assert lib.lse_evolve_batch(None, 1, None, 1, None, None) == lse.LSE_ERR_INVALID_ARG
    assert lib.lse_kernel_launches(None) == 0
    lib.lse_destroy(None)


def test_no_cpu_fallback_in_binding(lse):
    # the binding refuses to import without the library
    src = open(os.path.join(ROOT, "paper_1409_7474_gb300", "lse.py")).read()
    assert "raise ImportError" in src and "oracle" not in src


def test_strip_sums_layout_matches_header(lse, tmp_path):
    src = tmp_path / "strip.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "lse.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(lse_strip_sums),"
        " offsetof(lse_strip_sums, sum_w), offsetof(lse_strip_sums, sum_a),"
        " offsetof(lse_strip_sums, imin), offsetof(lse_strip_sums, fix_k),"
        " offsetof(lse_strip_sums, bands));return 0;}\n")
    exe = tmp_path / "strip"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    S = lse.StripSums
    assert vals == [ctypes.sizeof(S), S.sum_w.offset, S.sum_a.offset, S.imin.offset,
                    S.fix_k.offset, S.bands.offset]


@pytest.mark.parametrize("amax,npix", [(1.0, 65536), (0.7, 1000), (255.0, 8192 * 8192),
                                       (3.0, 5), (1e-30, 10 ** 6), (1e30, 4)])
def test_strip_scale_is_the_largest_safe_exponent(lse, amax, npix):
    # a host function: no context, no GPU.  k is the largest exponent with
    # max(npix, 32) * amax * 2^k <= 2^61
    k = lse.strip_scale(amax, npix)
    n = max(npix, 32)
    if -120 < k < 120:
        assert n * amax * 2.0 ** k <= 2.0 ** 61 < n * amax * 2.0 ** (k + 1)
    assert lse.strip_scale(0.0, npix) == 30 and lse.strip_scale(float("nan"), npix) == 30


def test_strip_calls_reject_a_null_context(lse):
    s = lse.StripSums()
    lib = lse.raw_library()
    assert lib.lse_strip_partials(None, None, 0, 4, 4, 1, 0, 4, None, None, 0,
                                  ctypes.byref(s), None) == lse.LSE_ERR_INVALID_ARG
    d = ctypes.c_double()
    assert lib.lse_strip_dmax(None, None, 0, 4, 4, 2, 0, 4, ctypes.byref(s), 15.0,
                              ctypes.byref(d), None) == lse.LSE_ERR_INVALID_ARG
    assert lib.lse_strip_step(None, None, 0, None, 4, 4, 1, None, 0, None, None, 0.0,
                              None, None) == lse.LSE_ERR_INVALID_ARG
