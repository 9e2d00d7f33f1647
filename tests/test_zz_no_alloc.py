"""hk_cross_section_noalloc: the cross section for callers that must not let
the library allocate device memory (scratch in a fixed device array).

Checked through the C ABI against hk_cross_section on the same inputs, twice
in a row (the fixed array keeps the previous call's contents, so the second
call shows that everything that must start at zero is cleared), in both
precisions and with a float output (whose overflow flag hk_noalloc_status
reads), plus the size and sortedness limits, and that a call leaves the
device's free memory unchanged while the library's pool cannot grow.  The file
name sorts last so that a run stopping at the first failure has run every
other test first.
"""
import numpy as np
import pytest

from parity import assert_sigma_close
from paper_2101_02005_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Q = synth.partition_function
QREF = float(Q(296.0))


@pytest.fixture(scope="module")
def hk():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2101_02005_gb300 import build
    build.build()
    from paper_2101_02005_gb300 import hk
    hk.lib()
    return hk


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_cross_section_twice(hk, prec):
    # config-1 shape (log-normal density, 0.1 cm^-1 grid, 25 cm^-1 cut) at
    # 1/1000 of its line count, then a second, different problem in a row
    for call, (scale, T, P) in enumerate([(1e-3, 1500.0, 1.0), (2e-4, 800.0, 0.03)]):
        w = synth.config(1, scale=scale)
        L = w.species[0]
        D = hk.DeviceLines.from_host(L)
        grid = hk.make_grid(*w.grid.astuple())
        st = hk.make_state(T, P, float(Q(T)))
        op = hk.make_opts(QREF, w.cut, prec, flags=hk.HK_SIGMA_F64)
        ref = hk.hk_cross_section(D, grid, st, op)
        out = torch.full_like(ref, 12345.0)      # stale contents must not leak into sigma
        hk.hk_cross_section_noalloc(D, grid, st, op, out)
        hk.hk_sync_status()
        assert_sigma_close(out.cpu().numpy(), ref.cpu().numpy(), f"noalloc call {call} prec={prec}")


def test_noalloc_limits(hk):
    L = synth.make_lines(100, 0.0, 50.0, 3, 18.0)
    D = hk.DeviceLines.from_host(L)
    st = hk.make_state(1000.0, 1.0, float(Q(1000.0)))
    op = hk.make_opts(QREF, 5.0)
    big = hk.make_grid(0.0, 1e-4, 3_000_000)         # FP32C needs ~24 MB > 16 MiB
    out = torch.empty(3_000_000, dtype=torch.float32, device="cuda")
    with pytest.raises(hk.HKError) as ei:
        hk.hk_cross_section_noalloc(D, big, st, op, out)
    assert ei.value.status == hk.HK_ESIZE
    U = synth.make_lines(100, 0.0, 50.0, 3, 18.0, sort=False)
    DU = hk.DeviceLines.from_host(U)
    small = hk.make_grid(0.0, 0.01, 5000)
    out = torch.empty(5000, dtype=torch.float32, device="cuda")
    with pytest.raises(hk.HKError) as ei:
        hk.hk_cross_section_noalloc(DU, small, st, op, out)
    assert ei.value.status == hk.HK_ENOTSUP


def test_noalloc_float_output_and_status(hk):
    # FP32C with a float sigma (no HK_SIGMA_F64): at 500 K the config-1 shape
    # stays in the float range; at 1500 K its hottest lines overflow it, which
    # hk_noalloc_status reports; the next call starts with a clear flag
    w = synth.config(1, scale=1e-3)
    D = hk.DeviceLines.from_host(w.species[0])
    grid = hk.make_grid(*w.grid.astuple())
    op = hk.make_opts(QREF, w.cut, hk.HK_FP32C)
    cool = hk.make_state(500.0, 1.0, float(Q(500.0)))
    hot = hk.make_state(1500.0, 1.0, float(Q(1500.0)))
    ref = hk.hk_cross_section(D, grid, cool, op)
    hk.hk_sync_status()
    assert ref.dtype == torch.float32
    for call in range(2):
        out = torch.full_like(ref, 12345.0)
        hk.hk_cross_section_noalloc(D, grid, cool, op, out)
        hk.hk_noalloc_status()
        assert_sigma_close(out.cpu().numpy().astype(np.float64),
                           ref.cpu().numpy().astype(np.float64), f"noalloc float call {call}")
    out = torch.empty_like(ref)
    hk.hk_cross_section_noalloc(D, grid, hot, op, out)
    with pytest.raises(hk.HKError) as ei:
        hk.hk_noalloc_status()
    assert ei.value.status == hk.HK_ERANGE
    hk.hk_noalloc_status()                           # cleared by the read
    hk.hk_cross_section_noalloc(D, grid, cool, op, out)
    hk.hk_noalloc_status()
    assert_sigma_close(out.cpu().numpy().astype(np.float64),
                       ref.cpu().numpy().astype(np.float64), "noalloc float after overflow")


def test_noalloc_allocates_nothing(hk, monkeypatch):
    # with the pool released and capped at 1 KB, hk_cross_section cannot get
    # its scratch (HK_ENOMEM) while hk_cross_section_noalloc still runs, and the
    # device's free memory is the same before and after two calls
    w = synth.config(1, scale=5e-4)
    D = hk.DeviceLines.from_host(w.species[0])
    grid = hk.make_grid(*w.grid.astuple())
    st = hk.make_state(1000.0, 0.3, float(Q(1000.0)))
    op = hk.make_opts(QREF, w.cut, hk.HK_FP32C, flags=hk.HK_SIGMA_F64)
    ref = hk.hk_cross_section(D, grid, st, op)
    outs = [torch.full_like(ref, -1.0) for _ in range(2)]
    hk.hk_cross_section_noalloc(D, grid, st, op, outs[0])    # loads the kernels
    torch.cuda.synchronize()
    hk.hk_release()
    monkeypatch.setenv("HK_POOL_LIMIT_MB", "0.001")
    with pytest.raises(hk.HKError) as ei:
        hk.hk_cross_section(D, grid, st, op)
    assert ei.value.status == hk.HK_ENOMEM
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for out in outs:
        hk.hk_cross_section_noalloc(D, grid, st, op, out)
    hk.hk_noalloc_status()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    for k, out in enumerate(outs):
        assert_sigma_close(out.cpu().numpy(), ref.cpu().numpy(), f"noalloc under pool cap {k}")
