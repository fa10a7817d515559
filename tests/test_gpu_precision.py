"""GPU parity of the reduced-cost operator arithmetics against the FP64 oracle.

df64 (FP32 pairs, about 48 significant bits; solution accumulated in FP64) is held to the
same bar as the native FP64 operator: 1e-12 relative L2 per step.  The FP32 operator's
error against the oracle is measured and bounded here (it is not an FP64-parity path):
3.3e-9 was measured after one step of the smooth vortex at CFL 0.1 (32^2, p=3); the bounds
are 2e-8 per step and 1e-6 after 50 steps.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_28710_gb300 import adg
from paper_2603_28710_gb300.inputs import random_state

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


@pytest.mark.parametrize("dim,n_elem,p", [(2, (5, 3), 1), (2, (5, 3), 4), (2, (4, 3), 7),
                                          (3, (3, 2, 2), 1), (3, (3, 2, 2), 3), (3, (2, 2, 2), 5)])
def test_df64_rhs_random_state(dim, n_elem, p):
    lo = (-5.0, -2.0, 0.0)[:dim]
    hi = (5.0, 3.0, 1.5)[:dim]
    s = adg.Solver(dim=dim, n_elem=n_elem, degree=p, lo=lo, hi=hi, dt=1e-3, precision="df64")
    o = O.Oracle(dim=dim, n_elem=n_elem, degree=p, lo=lo, hi=hi, dt=1e-3)
    u = random_state(s.shape, dim, seed=200 + p)
    assert rel(s.rhs(u), o.rhs(u)) < 1e-12


@pytest.mark.parametrize("flux,mode,L,rk", [("sync", "caa", 1, "ck45"), ("std", "caa", 3, "rk33"),
                                            ("at", "caa", 2, "ck45"), ("at_trace", "caa", 2, "rk22"),
                                            ("at", "random", 0, "ck45")])
def test_df64_steps_match_oracle(flux, mode, L, rk):
    kw = dict(P=(2, 3), max_delay=L, flux=flux, rk=rk, delay_mode=mode, random_delay_max=2,
              seed=11, dt=0.01)
    s = adg.Solver(n_elem=(8, 9), degree=2, precision="df64", **kw)
    o = O.Oracle(n_elem=(8, 9), degree=2, **kw)
    u0 = o.init_vortex(beta=3.0, x0=0.7, y0=-0.4)
    s.set_state(u0)
    o.set_state(u0)
    for n in range(12):
        s.step(1)
        o.step(1)
        assert rel(s.get_state(), o.get_state()) < 1e-12, f"step {n}"


def test_df64_large_vortex_steps():
    kw = dict(P=(8, 8), max_delay=3, flux="at", rk="ck45", dt=1.2e-4)
    s = adg.Solver(n_elem=(256, 256), degree=4, precision="df64", **kw)
    o = O.Oracle(n_elem=(256, 256), degree=4, **kw)
    u0 = o.init_vortex()
    s.set_state(u0)
    o.set_state(u0)
    s.step(1)
    o.step(1)
    assert rel(s.get_state(), o.get_state()) < 1e-12


def test_df64_3d_steps():
    kw = dict(P=(2, 2, 2), max_delay=2, flux="at", rk="rk33", dt=0.01)
    s = adg.Solver(dim=3, n_elem=(4, 4, 4), degree=3, lo=(0, 0, 0), hi=(2 * np.pi,) * 3,
                   precision="df64", **kw)
    o = O.Oracle(dim=3, n_elem=(4, 4, 4), degree=3, lo=(0, 0, 0), hi=(2 * np.pi,) * 3, **kw)
    u0 = o.init_tgv(0.1)
    s.set_state(u0)
    o.set_state(u0)
    for n in range(6):
        s.step(1)
        o.step(1)
        assert rel(s.get_state(), o.get_state()) < 1e-12, f"step {n}"


def test_df64_conserves():
    s = adg.Solver(n_elem=(32, 32), degree=4, P=(4, 4), max_delay=3, flux="at", dt=1e-3,
                   precision="df64")
    s.init_vortex()
    c0 = s.conservation()
    s.step(40)
    assert np.abs(s.conservation() - c0).max() < 1e-12 * np.abs(c0).max()


def test_fp32_error_bounded():
    kw = dict(P=(4, 4), max_delay=3, flux="at", rk="ck45")
    o0 = O.Oracle(n_elem=(32, 32), degree=3, dt=1.0)
    u0 = o0.init_vortex()
    dt = o0.dt_from_cfl(u0, 0.1, 0.0)
    s = adg.Solver(n_elem=(32, 32), degree=3, precision="fp32", dt=dt, **kw)
    o = O.Oracle(n_elem=(32, 32), degree=3, dt=dt, **kw)
    s.set_state(u0)
    o.set_state(u0)
    s.step(1)
    o.step(1)
    e1 = rel(s.get_state(), o.get_state())
    s.step(49)
    o.step(49)
    e50 = rel(s.get_state(), o.get_state())
    print(f"fp32 operator: relative L2 error after 1 step {e1:.2e}, after 50 steps {e50:.2e}")
    assert e1 < 2e-8
    assert e50 < 1e-6
    # FP32 operator, FP64 accumulation: both sides of a face use the one stored flux, so
    # the totals drift only by the FP32 rounding of each element's residual
    c = s.conservation()
    c0 = o0.conservation(u0)
    drift = np.abs(c - c0).max() / np.abs(c0).max()
    print(f"fp32 operator: conservation drift after 50 steps {drift:.2e}")
    assert drift < 1e-7


@pytest.mark.parametrize("flux,mode,rk", [("at", "caa", "rk22"), ("at", "caa", "rk33"),
                                          ("std", "caa", "ck45"), ("at_trace", "random", "ck45"),
                                          ("at", "random", "rk33")])
def test_fp32_steps_every_scheme(flux, mode, rk):
    # every update form of the FP32 volume kernel (2R stage 0 / later stages, 2N) and its
    # staged operands against the FP64 oracle
    kw = dict(P=(4, 4), max_delay=3, flux=flux, rk=rk, delay_mode=mode, random_delay_max=2,
              seed=99)
    o0 = O.Oracle(n_elem=(16, 12), degree=3, dt=1.0)
    u0 = o0.init_vortex()
    dt = o0.dt_from_cfl(u0, 0.1, 0.0)
    s = adg.Solver(n_elem=(16, 12), degree=3, precision="fp32", dt=dt, **kw)
    o = O.Oracle(n_elem=(16, 12), degree=3, dt=dt, **kw)
    s.set_state(u0)
    o.set_state(u0)
    s.step(1)
    o.step(1)
    e1 = rel(s.get_state(), o.get_state())
    s.step(19)
    o.step(19)
    e20 = rel(s.get_state(), o.get_state())
    print(f"fp32 {flux}/{mode}/{rk}: relative L2 error after 1 step {e1:.2e}, after 20 {e20:.2e}")
    assert e1 < 2e-8
    assert e20 < 5e-7


@pytest.mark.parametrize("dim,n_elem,p", [(2, (5, 3), 2), (2, (7, 4), 5), (3, (3, 2, 2), 3)])
def test_fp32_rhs_random_state(dim, n_elem, p):
    # adg_rhs in the FP32 operator: the output as an increment over a CFL-limited step
    lo, hi = (-5.0,) * dim, (5.0,) * dim
    s = adg.Solver(dim=dim, n_elem=n_elem, degree=p, lo=lo, hi=hi, dt=1e-3, precision="fp32")
    o = O.Oracle(dim=dim, n_elem=n_elem, degree=p, lo=lo, hi=hi, dt=1e-3)
    u = random_state(s.shape, dim, seed=31 + p)
    kg = s.rhs(u)
    ko = o.rhs(u)
    dt = o.dt_from_cfl(u, 0.1, 0.0)
    inc = np.linalg.norm((kg - ko) * dt) / np.linalg.norm(u)
    print(f"fp32 rhs {dim}D p={p}: increment error {inc:.2e}")
    assert inc < 1e-7


def test_fp32_3d_steps():
    kw = dict(P=(2, 2, 2), max_delay=2, flux="at", rk="ck45", dt=0.01)
    dim, n_elem, p = 3, (4, 4, 4), 2
    lo, hi = (0.0,) * 3, (2 * np.pi,) * 3
    s = adg.Solver(dim=dim, n_elem=n_elem, degree=p, lo=lo, hi=hi, precision="fp32", **kw)
    o = O.Oracle(dim=dim, n_elem=n_elem, degree=p, lo=lo, hi=hi, **kw)
    u0 = o.init_tgv(0.3)
    s.set_state(u0)
    o.set_state(u0)
    s.step(6)
    o.step(6)
    e6 = rel(s.get_state(), o.get_state())
    print(f"fp32 3D Taylor-Green 4^3 p=2, 6 AT steps: relative L2 error {e6:.2e}")
    assert e6 < 1e-6
