"""The element path (one launch per RK stage; every element evaluates the numerical flux on
each of its own faces from the stored traces) against the split path and the oracle.

Both paths evaluate a face's flux with the same code from the same two stored traces, and
the element path lifts it in the same order, so the results are equal bit for bit in every
arithmetic (FP64, FP32 pairs, FP32) and the face terms still cancel exactly across each
face.  Subdomain faces are evaluated by both of their elements; only the low element
stores ring levels, and no stage reads the level it stores, so the two evaluations read
the same ring entries.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_28710_gb300 import adg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_28710_gb300 import build
    build.build()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def run(path, precision, dim, n_elem, degree, steps, tgv=False, **kw):
    lo = (0.0,) * 3 if tgv else (-5.0,) * dim
    hi = (2 * np.pi,) * 3 if tgv else (5.0,) * dim
    s = adg.Solver(dim=dim, n_elem=n_elem, degree=degree, lo=lo, hi=hi, precision=precision,
                   kernel_path=path, **kw)
    if tgv:
        s.init_tgv(0.1)
    else:
        s.init_vortex(beta=3.0, x0=0.7, y0=-0.4)
    c0 = s.conservation()
    s.step(steps)
    u = s.get_state()
    c1 = s.conservation()
    s.close()
    return u, c0, c1


CASES_2D = [((16, 16), 4), ((8, 9), 2), ((13, 7), 3), ((5, 3), 4), ((12, 8), 1), ((8, 4), 5),
            ((6, 4), 6), ((4, 6), 7), ((1, 4), 3)]
MODES = [("sync", "caa", 1, "ck45"), ("at", "caa", 2, "ck45"), ("std", "caa", 3, "rk33"),
         ("at_trace", "caa", 2, "rk22"), ("at", "random", 0, "ck45"),
         ("std", "random", 0, "rk22")]


@pytest.mark.parametrize("precision", ["fp64", "df64", "fp32"])
@pytest.mark.parametrize("n_elem,p", CASES_2D)
@pytest.mark.parametrize("flux,mode,L,rk", MODES)
def test_element_equals_split_bitwise_2d(precision, n_elem, p, flux, mode, L, rk):
    P = tuple(2 if n % 2 == 0 else 1 for n in n_elem)
    kw = dict(P=P, max_delay=L, flux=flux, rk=rk, delay_mode=mode, random_delay_max=2,
              seed=20260301, dt=0.004)
    a, _, _ = run("split", precision, 2, n_elem, p, 9, **kw)
    b, c0, c1 = run("element", precision, 2, n_elem, p, 9, **kw)
    assert np.array_equal(a, b), rel(b, a)
    if precision != "fp32":
        assert np.abs(c1 - c0).max() < 1e-12 * np.abs(c0).max()


@pytest.mark.parametrize("precision", ["fp64", "df64", "fp32"])
@pytest.mark.parametrize("n_elem,p", [((4, 4, 4), 3), ((3, 2, 2), 2), ((5, 3, 4), 2),
                                      ((4, 4, 2), 1), ((2, 2, 2), 4), ((2, 2, 1), 5),
                                      ((1, 2, 3), 3)])
@pytest.mark.parametrize("flux,mode,L,rk", [("at", "caa", 2, "ck45"), ("at_trace", "random", 0, "rk33"),
                                           ("std", "caa", 4, "ck45")])
def test_element_equals_split_bitwise_3d(precision, n_elem, p, flux, mode, L, rk):
    P = tuple(2 if n % 2 == 0 else 1 for n in n_elem)
    kw = dict(P=P, max_delay=L, flux=flux, rk=rk, delay_mode=mode, random_delay_max=2,
              seed=7, dt=0.004)
    a, _, _ = run("split", precision, 3, n_elem, p, 7, tgv=True, **kw)
    b, c0, c1 = run("element", precision, 3, n_elem, p, 7, tgv=True, **kw)
    assert np.array_equal(a, b), rel(b, a)
    if precision != "fp32":
        assert np.abs(c1 - c0).max() < 1e-12 * np.abs(c0).max()


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_element_path_matches_oracle_at_the_256_configuration_settings(precision):
    # 2D p=4, N_p=4 (five levels), L=3, 8x8 subdomains, CK4(5) on 32^2: two schedule
    # cycles, the increment of every step compared element by element
    kw = dict(P=(8, 8), max_delay=3, flux="at", rk="ck45", dt=2e-3)
    s = adg.Solver(n_elem=(32, 32), degree=4, precision=precision, kernel_path="element", **kw)
    o = O.Oracle(n_elem=(32, 32), degree=4, **kw)
    u0 = o.init_vortex()
    s.set_state(u0)
    o.set_state(u0)
    wg0, wo0 = u0.copy(), u0.copy()
    eps = 2.0 ** -53 if precision == "fp64" else 2.0 ** -48
    for n in range(16):
        s.step(1)
        o.step(1)
        wg1, wo1 = s.get_state(), o.get_state()
        dg, do = wg1 - wg0, wo1 - wo0
        scale = np.abs(wo1).max()
        assert np.abs(dg - do).max() <= 1e-11 * np.abs(do).max() + 64 * 5 * eps * scale, n
        assert rel(wg1, wo1) < 1e-12, n
        wg0, wo0 = wg1, wo1
    s.close()


def test_element_path_3d_matches_oracle():
    # 3D Taylor-Green p=3 (N_p=3), L=4, 2x2x2 subdomains on 4^3: ten steps
    kw = dict(dim=3, n_elem=(4, 4, 4), lo=(0.0,) * 3, hi=(2 * np.pi,) * 3, degree=3,
              P=(2, 2, 2), max_delay=4, flux="at", rk="ck45", dt=0.01)
    s = adg.Solver(kernel_path="element", **kw)
    o = O.Oracle(**kw)
    u0 = o.init_tgv(0.1)
    s.set_state(u0)
    o.set_state(u0)
    for n in range(10):
        s.step(1)
        o.step(1)
        assert rel(s.get_state(), o.get_state()) < 1e-12, n
    s.close()


def test_element_checkpoint_and_trace_log_equal_split():
    # the element path keeps every face trace, so checkpoints move between the paths and
    # the subdomain-trace log records the same values
    import torch
    kw = dict(n_elem=(16, 16), degree=3, P=(4, 4), max_delay=3, flux="at", rk="ck45", dt=3e-3)
    runs = {}
    for path in ("split", "element"):
        s = adg.Solver(kernel_path=path, **kw)
        s.init_vortex()
        s.step(5)
        ck = s.checkpoint()
        rec = s.set_trace_log(None, 0)
        log = torch.zeros((10, rec), dtype=torch.float64, device="cuda")
        s.set_trace_log(log, 10)
        s.step(2)
        s.set_trace_log(None, 0)
        s.step(4)
        runs[path] = (ck, s.get_state(), log.cpu().numpy())
        s.close()
    assert np.array_equal(runs["split"][0], runs["element"][0])
    assert np.array_equal(runs["split"][1], runs["element"][1])
    assert np.array_equal(runs["split"][2], runs["element"][2])
    # a split-path handle continues the element path's checkpoint exactly
    b = adg.Solver(kernel_path="split", **kw)
    b.restore(runs["element"][0])
    b.set_trace_log(None, 0)
    b.step(6)
    assert np.array_equal(b.get_state(), runs["element"][1])
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "df64", "fp32"])
def test_element_equals_split_at_full_size(precision):
    # the 256^2 p=4 workload (8x8 subdomains, CAA L=3, AT, CK4(5)): one schedule cycle
    kw = dict(n_elem=(256, 256), degree=4, P=(8, 8), max_delay=3, flux="at", rk="ck45",
              cfl=0.1, precision=precision)
    out = []
    for path in ("split", "element"):
        s = adg.Solver(kernel_path=path, **kw)
        s.init_vortex()
        s.step(8)
        out.append(s.get_state())
        s.close()
    assert np.array_equal(out[0], out[1])


def test_element_equals_split_3d_full_size_fp32():
    # the 64^3 p=3 Taylor-Green workload (8x8x8 subdomains, CAA L=4, AT, CK4(5)): 4 steps
    kw = dict(dim=3, n_elem=(64, 64, 64), lo=(0.0,) * 3, hi=(2 * np.pi,) * 3, degree=3,
              P=(8, 8, 8), max_delay=4, flux="at", rk="ck45", cfl=0.1, precision="fp32")
    out = []
    for path in ("split", "element"):
        s = adg.Solver(kernel_path=path, **kw)
        s.init_tgv(0.1)
        s.step(4)
        out.append(s.get_state())
        s.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("precision,path,flux,expect_flux_launches", [
    ("fp32", "auto", "at", False), ("fp64", "auto", "at", True), ("df64", "auto", "at", True),
    ("fp64", "element", "at", False), ("fp32", "split", "at", True),
    ("fp32", "element", "sync", False)])
def test_path_selection(precision, path, flux, expect_flux_launches):
    # the default takes the element path for the FP32 operator and the split path for the
    # FP64 and pair operators; an explicit path is taken as given
    s = adg.Solver(n_elem=(8, 8), degree=2, P=(2, 2), max_delay=2, flux=flux, rk="ck45",
                   dt=1e-3, precision=precision, kernel_path=path)
    s.init_vortex()
    s.set_profiling(True)
    s.step(2)
    prof = s.get_profile()
    s.set_profiling(False)
    s.close()
    assert prof["vol"][1] == 10
    assert (prof["flux"][1] > 0) == expect_flux_launches
