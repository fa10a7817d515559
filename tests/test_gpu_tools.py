"""The package's command-line helpers on the GPU: the profiler driver runs a small case of
each operator form in 2D and 3D and leaves a finite state."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_28710_gb300 import build
    build.build()


@pytest.mark.parametrize("precision", ["fp64", "df64", "fp32"])
@pytest.mark.parametrize("dim", [2, 3])
def test_profile_case_runs(dim, precision, capsys):
    from paper_2603_28710_gb300 import profile_case
    profile_case.main(["--dim", str(dim), "--n", "8", "--degree", "2", "--P", "2", "--L", "2",
                       "--steps", "3", "--precision", precision])
    out = capsys.readouterr().out
    assert "finite=True" in out and f"dim={dim}" in out


def test_peak_probe_rates_are_plausible():
    # GB300 nominal: FP64 1.25 TFLOP/s, FP32 about 75; the probe must land near them and
    # order them (FP32 far above FP64)
    from paper_2603_28710_gb300 import adg
    f64, ms64, mhz = adg.measure_peak("fp64_fma")
    f32, _, _ = adg.measure_peak("fp32_fma")
    mma, _, _ = adg.measure_peak("fp64_mma")
    both, _, _ = adg.measure_peak("fp64_fma+mma")
    assert 0.3 < f64 < 3.0 and ms64 > 5.0
    assert 500.0 < mhz < 3000.0
    assert 20.0 < f32 < 150.0 and f32 > 10 * f64
    assert mma > 0.0 and both > 0.0


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    # the fused and element-path kernels' mbarrier wait, on a barrier nothing arrives at:
    # every thread gives up after the limit (about 1 ms here), and the device is fine after
    from paper_2603_28710_gb300 import adg
    limit = 2_000_000
    n, cycles = adg.probe_wait(limit)
    assert n == 128
    assert limit < cycles < 4 * limit + 1_000_000
    s = adg.Solver(n_elem=(8, 8), degree=2, P=(2, 2), max_delay=2, flux="at", rk="ck45",
                   dt=1e-3, precision="fp32", kernel_path="element")
    s.init_vortex()
    s.step(3)
    assert s.check_finite()
    s.get_state()                       # the element path's error flag is clear
    s.close()
