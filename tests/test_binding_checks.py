"""Host-side checks of the Python binding (no GPU): the output-tensor checks
that stop the library from writing past a caller's buffer, the output type
the options select, and the loud failure when the library is not built."""
import pytest

torch = pytest.importorskip("torch")

from paper_2101_02005_gb300 import hk  # noqa: E402


def test_sigma_dtype_follows_the_options():
    assert hk.sigma_dtype(hk.make_opts(1.0, 25.0, hk.HK_FP32C)) == torch.float32
    assert hk.sigma_dtype(hk.make_opts(1.0, 25.0, hk.HK_FP32C, flags=hk.HK_SIGMA_F64)) == \
        torch.float64
    assert hk.sigma_dtype(hk.make_opts(1.0, 25.0, hk.HK_FP64)) == torch.float64


@pytest.mark.parametrize("bad, what", [
    (torch.empty(100, dtype=torch.float32), "dtype"),
    (torch.empty(99, dtype=torch.float64), "elements"),
    (torch.empty(200, dtype=torch.float64)[::2], "contiguous"),
])
def test_output_checks_reject_a_buffer_the_library_would_overrun(bad, what):
    with pytest.raises(ValueError, match=what):
        hk._check_out("hk_cross_section", bad, 100, torch.float64, host_ok=True)


def test_output_checks_want_device_memory_unless_host_is_allowed():
    t = torch.empty(100, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA"):
        hk._check_out("hk_cross_section", t, 100, torch.float64)
    hk._check_out("hk_cross_section_host", t, 100, torch.float64, host_ok=True)
    # a larger buffer than needed is accepted
    hk._check_out("hk_cross_section_host", torch.empty(101, dtype=torch.float64), 100,
                  torch.float64, host_ok=True)


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(hk, "_lib", None)
    monkeypatch.setattr(hk, "LIB_PATH", str(tmp_path / "libhk.so"))
    with pytest.raises(ImportError, match="not built"):
        hk.lib()


def _cpu_lines(n=4):
    f = lambda: torch.zeros(n, dtype=torch.float32)  # noqa: E731
    return hk.DeviceLines(torch.zeros(n, dtype=torch.float64), f(), f(), f(), f(), 18.0)


@pytest.mark.parametrize("precision, flags, out_dtype", [
    (hk.HK_FP64, 0, torch.float32),
    (hk.HK_FP32C, hk.HK_SIGMA_F64, torch.float32),
    (hk.HK_FP32C, 0, torch.float64),
])
def test_entry_points_check_sigma_before_calling_the_library(monkeypatch, precision, flags,
                                                             out_dtype):
    """A sigma of the wrong element type never reaches the library: the
    wrappers raise before loading or calling it."""
    def no_library():
        raise AssertionError("the library was called")
    monkeypatch.setattr(hk, "lib", no_library)
    grid = hk.make_grid(0.0, 0.1, 100)
    state = hk.make_state(1500.0, 1.0, 1.0)
    opts = hk.make_opts(1.0, 25.0, precision, flags=flags)
    out = torch.empty(100, dtype=out_dtype)
    for fn in (hk.hk_cross_section, hk.hk_cross_section_noalloc):
        with pytest.raises(ValueError, match="dtype"):
            fn(_cpu_lines(), grid, state, opts, out)
    with pytest.raises(ValueError, match="dtype"):
        hk.hk_cross_section_host(_cpu_lines(), grid, state, opts, out)
