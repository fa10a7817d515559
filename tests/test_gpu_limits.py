"""The largest settings the library accepts, against the oracle.

* degree 7 (the largest 2D degree) with the AT flux at its default N_p = 7 (eight stored
  levels) and the CAA schedule at its largest delay L = 15 (a cycle of 23 steps: 8
  communication steps, then delays k = 1..15, the largest AT weight table);
* the random-delay mode at its largest delay bound, 15 (ring depth 15 + N_p + 1);
* 3D at its largest degree, 5.
The AT weights at k = 15 with N_p = 7 alternate in sign with magnitudes up to about 7e6
(Lagrange extrapolation far outside the stored levels), so the weighted sums cancel: the
FP64 rounding of the two sides' different summation orders reaches about 1e-9 of a flux
on those steps, and the states are compared at 1e-10 instead of 1e-12.  Schedules are
compared bit for bit.
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


def test_degree7_at_largest_caa_delay():
    kw = dict(n_elem=(4, 6), degree=7, P=(2, 2), max_delay=15, flux="at", rk="ck45", dt=2e-3)
    s, o = adg.Solver(**kw), O.Oracle(**kw)
    u0 = o.init_vortex(beta=2.0)
    s.set_state(u0)
    o.set_state(u0)
    worst = 0.0
    for n in range(24):
        s.step(1)
        o.step(1)
        worst = max(worst, rel(s.get_state(), o.get_state()))
        assert worst < 1e-10, (n, worst)
    comm_g, k_g, _ = s.schedule(0, 24)
    comm_o, k_o, _ = O.schedule("at", "caa", 15, 7, (2, 2), 2, 0, 0, 0, 24)
    assert np.array_equal(comm_g, comm_o) and np.array_equal(k_g, k_o)
    assert k_o.max() == 15
    c = O.at_coeffs(7, 15.0)
    assert np.abs(c).max() > 1e5          # the cancellation the tolerance allows for
    s.close()


@pytest.mark.parametrize("flux", ["std", "at"])
def test_random_delays_up_to_15(flux):
    kw = dict(n_elem=(6, 4), degree=2, P=(3, 2), max_delay=1, flux=flux, rk="rk33",
              delay_mode="random", random_delay_max=15, seed=99, dt=2e-3)
    s, o = adg.Solver(**kw), O.Oracle(**kw)
    u0 = o.init_vortex(beta=2.0)
    s.set_state(u0)
    o.set_state(u0)
    for n in range(40):
        s.step(1)
        o.step(1)
        assert rel(s.get_state(), o.get_state()) < 1e-10, n
    _, _, d_g = s.schedule(0, 40)
    _, _, d_o = O.schedule(flux, "random", 1, 2, (3, 2), 2, 99, 15, 0, 40)
    assert np.array_equal(d_g, d_o) and d_o.max() >= 12
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_3d_largest_degree(precision):
    kw = dict(dim=3, n_elem=(2, 2, 2), degree=5, lo=(0, 0, 0), hi=(2 * np.pi,) * 3, P=(2, 1, 2),
              max_delay=2, flux="at", rk="ck45", dt=2e-3)
    s = adg.Solver(precision=precision, **kw)
    o = O.Oracle(**kw)
    u0 = o.init_tgv(0.1)
    s.set_state(u0)
    o.set_state(u0)
    for n in range(6):
        s.step(1)
        o.step(1)
        assert rel(s.get_state(), o.get_state()) < 1e-12, n
    s.close()
