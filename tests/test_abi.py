"""The C-ABI library loads and exports every entry point of include/hk.h;
host-side argument checks and constants need no GPU."""
import ctypes
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hk():
    from paper_2101_02005_gb300 import build
    build.build()
    from paper_2101_02005_gb300 import hk
    hk.lib()
    return hk


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hk.h")).read()
    return sorted(set(re.findall(r"^(?:int|const char \*)\s*(hk_\w+)\(", src, re.M)))


def test_every_declared_symbol_is_exported(hk):
    names = declared_symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(hk.lib(), n), n
        assert n in hk.EXPORTS, n


def test_constants_match_paper_and_oracle(hk):
    import oracle
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    d = hk.hk_constants()
    assert d["k_B"] == g["k_B"]["value"] and d["c"] == g["c"]["value"]
    o = oracle.constants()
    for k in d:
        assert d[k] == o[k], k


def test_strerror_and_version(hk):
    L = hk.lib()
    assert L.hk_strerror(0) == b"ok" and b"invalid" in L.hk_strerror(1)
    assert L.hk_version() >= 100


def test_invalid_arguments_rejected_on_host(hk):
    L = hk.lib()
    lines = hk.hk_lines(1, 2, None, None, 3, 4, 5, 10, 18.0, 0, 1)
    grid = hk.make_grid(0.0, 0.1, 100)
    st = hk.make_state(1000.0, 1.0, 3000.0)
    op = hk.make_opts(500.0, 25.0)
    b = ctypes.byref
    assert L.hk_cross_section(None, b(grid), b(st), b(op), 1, None) == hk.HK_EINVAL
    bad = hk.make_grid(0.0, -0.1, 100)
    assert L.hk_cross_section(b(lines), b(bad), b(st), b(op), 1, None) == hk.HK_EINVAL
    bad = hk.make_grid(0.0, 0.1, 0)
    assert L.hk_cross_section(b(lines), b(bad), b(st), b(op), 1, None) == hk.HK_EINVAL
    bst = hk.make_state(-1.0, 1.0, 3000.0)
    assert L.hk_cross_section(b(lines), b(grid), b(bst), b(op), 1, None) == hk.HK_EINVAL
    bst = hk.make_state(1000.0, -1.0, 3000.0)
    assert L.hk_cross_section(b(lines), b(grid), b(bst), b(op), 1, None) == hk.HK_EINVAL
    bop = hk.make_opts(500.0, float("nan"))
    assert L.hk_cross_section(b(lines), b(grid), b(st), b(bop), 1, None) == hk.HK_EINVAL
    bop = hk.make_opts(500.0, 25.0, precision=7)
    assert L.hk_cross_section(b(lines), b(grid), b(st), b(bop), 1, None) == hk.HK_EINVAL
    nl = hk.hk_lines(1, 2, None, None, 3, 4, 5, -1, 18.0, 0, 1)
    assert L.hk_cross_section(b(nl), b(grid), b(st), b(op), 1, None) == hk.HK_EINVAL
    nm = hk.hk_lines(1, None, None, None, 3, 4, 5, 10, 18.0, 0, 1)  # S-mode without S_ref
    assert L.hk_cross_section(b(nm), b(grid), b(st), b(op), 1, None) == hk.HK_EINVAL
    assert L.hk_cross_section(b(lines), b(grid), b(st), b(op), None, None) == hk.HK_EINVAL
    out = ctypes.c_size_t(0)
    assert L.hk_workspace_size(2, b(lines), 1, 1, b(grid), b(op), b(out)) == hk.HK_EINVAL
    assert L.hk_constants(None) == hk.HK_EINVAL


def test_new_options_validated_on_host(hk):
    """Cut modes, profiles, flags, the self pressure and the tuning setter are
    checked before any device work."""
    L = hk.lib()
    lines = hk.hk_lines(1, 2, None, None, 3, 4, 5, 10, 18.0, 0, 1)
    grid = hk.make_grid(0.0, 0.1, 100)
    st = hk.make_state(1000.0, 1.0, 3000.0)
    b = ctypes.byref
    for bop in (hk.make_opts(500.0, 0.0, cut_mode=hk.HK_CUT_DOPPLER),       # factor must be > 0
                hk.make_opts(500.0, -3.0, cut_mode=hk.HK_CUT_LORENTZ),
                hk.make_opts(500.0, 25.0, cut_mode=9),
                hk.make_opts(500.0, 25.0, profile=4),
                hk.make_opts(500.0, 25.0, profile=-1),
                hk.make_opts(500.0, 25.0, flags=8)):
        assert L.hk_cross_section(b(lines), b(grid), b(st), b(bop), 1, None) == hk.HK_EINVAL
        assert L.hk_cross_section_host(b(lines), b(grid), b(st), b(bop), 1, 0, None) == hk.HK_EINVAL
    op = hk.make_opts(500.0, 25.0)
    bst = hk.make_state(1000.0, 1.0, 3000.0, P_self=-0.1)
    assert L.hk_cross_section(b(lines), b(grid), b(bst), b(op), 1, None) == hk.HK_EINVAL
    assert L.hk_cross_section_host(b(lines), b(grid), b(st), b(op), 1, -5, None) == hk.HK_EINVAL
    assert L.hk_set_tuning(hk.HK_FP32C, 8, 0) == hk.HK_EINVAL
    assert L.hk_set_tuning(7, 2048, 0) == hk.HK_EINVAL
    assert L.hk_set_tuning(hk.HK_FP32C, 2048, 1536) == hk.HK_EINVAL   # tile widths: 1024, 2048
    assert L.hk_set_tuning(hk.HK_FP64, 2048, 1024) == hk.HK_EINVAL    # FP64 tiles: 512
    v = ctypes.c_int(0)
    assert L.hk_tuning(7, b(v), None) == hk.HK_EINVAL


def test_other_entry_points_validate_on_host(hk):
    """The instrumentation, no-allocation, batched, adjoint and accumulate
    entry points reject bad arguments before any device work."""
    L = hk.lib()
    b = ctypes.byref
    lines = hk.hk_lines(1, 2, None, None, 3, 4, 5, 10, 18.0, 0, 1)
    unsorted = hk.hk_lines(1, 2, None, None, 3, 4, 5, 10, 18.0, 0, 0)
    grid = hk.make_grid(0.0, 0.1, 100)
    st = hk.make_state(1000.0, 1.0, 3000.0)
    op = hk.make_opts(500.0, 25.0)
    assert L.hk_count_pairs(b(lines), b(grid), b(st), b(op), None, None) == hk.HK_EINVAL
    assert L.hk_count_ring_pairs(b(lines), b(grid), b(st), b(op), None, None) == hk.HK_EINVAL
    ms, n = ctypes.c_double(0), ctypes.c_int64(0)
    assert L.hk_profile(2, b(ms), b(n)) == hk.HK_EINVAL
    v = ctypes.c_double(0)
    for kind, target, out in ((5, 100.0, b(v)), (-1, 100.0, b(v)), (0, 0.0, b(v)),
                              (0, 1e5, b(v)), (0, float("nan"), b(v)), (0, 100.0, None)):
        assert L.hk_measure_peak(kind, target, out, None) == hk.HK_EINVAL
    # no-allocation entry: an output is required and the list must be sorted
    assert L.hk_cross_section_noalloc(b(lines), b(grid), b(st), b(op), None, None) == hk.HK_EINVAL
    assert L.hk_cross_section_noalloc(b(unsorted), b(grid), b(st), b(op), 1, None) == \
        hk.HK_ENOTSUP
    # batched: counts, outputs and precision
    two = (hk.hk_lines * 2)(lines, lines)
    sts = (hk.hk_state * 2)(st, st)
    for ns, nt in ((0, 2), (2, 0), (-1, 2)):
        assert L.hk_cross_section_batched(two, ns, sts, nt, b(grid), b(op), 1, 1, 1 << 30,
                                          None) == hk.HK_EINVAL
    assert L.hk_cross_section_batched(two, 2, sts, 2, b(grid), b(op), None, 1, 1 << 30,
                                      None) == hk.HK_EINVAL
    op64 = hk.make_opts(500.0, 25.0, precision=hk.HK_FP64)
    assert L.hk_cross_section_batched(two, 2, sts, 2, b(grid), b(op64), 1, 1, 1 << 30,
                                      None) == hk.HK_ENOTSUP
    # adjoint: points, upstream gradient and outputs; options it does not cover
    assert L.hk_cross_section_backward(b(lines), b(grid), sts, 0, b(op), 1, 1, 1, 1, 1, 1,
                                       1 << 30, None) == hk.HK_EINVAL
    assert L.hk_cross_section_backward(b(lines), b(grid), sts, 2, b(op), None, 1, 1, 1, 1, 1,
                                       1 << 30, None) == hk.HK_EINVAL
    assert L.hk_cross_section_backward(b(lines), b(grid), sts, 2, b(op), 1, 1, 1, None, 1, 1,
                                       1 << 30, None) == hk.HK_EINVAL
    opp = hk.make_opts(500.0, 25.0, flags=hk.HK_REMOVE_PLINTH)
    assert L.hk_cross_section_backward(b(lines), b(grid), sts, 2, b(opp), 1, 1, 1, 1, 1, 1,
                                       1 << 30, None) == hk.HK_ENOTSUP
    # the bare accumulate: line count, precision, cut and pointers
    assert L.hk_voigt_accumulate(1, 2, 3, 4, -1, b(grid), 25.0, 5, hk.HK_FP32C, None) == \
        hk.HK_EINVAL
    assert L.hk_voigt_accumulate(1, 2, 3, 4, 10, b(grid), 25.0, 5, 7, None) == hk.HK_EINVAL
    assert L.hk_voigt_accumulate(1, 2, 3, 4, 10, b(grid), float("inf"), 5, hk.HK_FP32C,
                                 None) == hk.HK_EINVAL
    assert L.hk_voigt_accumulate(None, 2, 3, 4, 10, b(grid), 25.0, 5, hk.HK_FP32C, None) == \
        hk.HK_EINVAL
    assert L.hk_voigt_accumulate(1, 2, 3, 4, 10, b(grid), 25.0, None, hk.HK_FP32C, None) == \
        hk.HK_EINVAL
