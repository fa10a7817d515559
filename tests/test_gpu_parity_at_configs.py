"""GPU parity at the benchmarked delay configurations, step by step, on the increments.

The benchmark runs the AT flux of Algorithm 3 with N_p = 4 (five stored flux levels, Eq. 14
with the weights of Eq. 15 at r = 1) on the 2D vortex and N_p = 3 on the 3D Taylor-Green
vortex.  Here the CUDA path and the oracle advance together through whole schedule cycles,
so every delayed (non-communication) step -- the ring read with the stage weights c~(k_m)
-- is compared, not only the communication steps that fill the ring.

What is compared is the increment of each step, dw = w(n+1) - w(n), element by element,
because the state itself hides errors of the increment: over one CFL-limited step the
increment is about 1e-4 of the state.  The comparison has a floor that no correct pair of
implementations can beat: each side adds its s stage increments to w in FP64, so each
increment carries up to s roundings of ulp(w)/2 per side (two per stage where the
FP32-pair operator adds its (hi, lo) increment: bound 4 s eps |w| for the difference of the
two sides), and the two states entering the step already differ by what the earlier steps
left (propagated through one step with a factor of about one at CFL 0.1).  Node by node the
operator adds its own floor: its weak derivative cancels terms far larger than its result
(the uniform part of the pressure, the background energy), and the rounding of those terms
reaches the increment of a node at a few tens of eps |w| (measured on GB300: up to about
20 s eps max|w| in 2D and 3D).
Bounds (eps = 2^-53):
  relative L2:  |dw_g - dw_o| <= 1e-12 |dw_o| + 4 s eps |w| + |w_g(n) - w_o(n)|
  max norm:     max|dw_g - dw_o| <= 1e-11 max|dw_o| + 64 s eps max|w| + max|w_g(n) - w_o(n)|
and, independently of the floor, the relative L2 difference of the increments stays below
1e-9.  The FP32-pair operator computes in about 48-bit arithmetic: its floors take
eps = 2^-48 and its cap is 1e-8.  (A fixed 1e-12 relative bound on the increments cannot hold: on the Taylor-Green
vortex at Mach 0.1 the energy is about 180 while a step changes the state by about 1e-4,
so one rounding of w alone is about 2e-10 of the increment.)  A sensitivity check shows that the comparison sees the delayed-face rule: the
oracle with a lower-order AT weight set differs from the CUDA increments over one cycle by
orders of magnitude more than the bound.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_28710_gb300 import adg

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_28710_gb300 import build
    build.build()


def cfl_dt(dim, n_elem, degree, lo, hi, tgv):
    o = O.Oracle(dim=dim, n_elem=n_elem, degree=degree, lo=lo, hi=hi, dt=1.0)
    u0 = o.init_tgv(0.1) if tgv else o.init_vortex()
    return u0, o.dt_from_cfl(u0, 0.1, 0.0)


def increment_bounds(wg0, wo0, wg1, wo1, stages, rel_cap=1e-9, eps=EPS):
    """(ok, report) for one step's increments against the bounds of the module docstring."""
    dg, do = wg1 - wg0, wo1 - wo0
    diff = dg - do
    state_l2 = np.linalg.norm(wg0 - wo0)
    state_max = np.abs(wg0 - wo0).max()
    l2 = np.linalg.norm(diff)
    l2_bound = 1e-12 * np.linalg.norm(do) + 4 * stages * eps * np.linalg.norm(wo0) + state_l2
    mx = np.abs(diff).max()
    mx_bound = 1e-11 * np.abs(do).max() + 64 * stages * eps * np.abs(wo0).max() + state_max
    rel = l2 / np.linalg.norm(do)
    ok = l2 <= l2_bound and mx <= mx_bound and rel < rel_cap
    return ok, dict(rel=rel, l2=l2, l2_bound=l2_bound, max=mx, max_bound=mx_bound)


def run_pair(dim, n_elem, degree, steps, precision="fp64", tgv=False, **kw):
    lo = (0.0,) * 3 if tgv else (-5.0,) * dim
    hi = (2 * np.pi,) * 3 if tgv else (5.0,) * dim
    u0, dt = cfl_dt(dim, n_elem, degree, lo, hi, tgv)
    s = adg.Solver(dim=dim, n_elem=n_elem, degree=degree, lo=lo, hi=hi, dt=dt,
                   precision=precision, **kw)
    o = O.Oracle(dim=dim, n_elem=n_elem, degree=degree, lo=lo, hi=hi, dt=dt, **kw)
    s.set_state(u0)
    o.set_state(u0)
    stages = 5 if kw.get("rk", "ck45") == "ck45" else (3 if kw["rk"] == "rk33" else 2)
    wg0, wo0 = u0.copy(), u0.copy()
    reports = []
    for n in range(steps):
        s.step(1)
        o.step(1)
        wg1, wo1 = s.get_state(), o.get_state()
        ok, rep = increment_bounds(wg0, wo0, wg1, wo1, stages,
                                   rel_cap=1e-8 if precision == "df64" else 1e-9,
                                   eps=2.0 ** -48 if precision == "df64" else EPS)
        rep["step"] = n
        reports.append(rep)
        assert ok, " ".join(f"{k}={v:.3e}" for k, v in rep.items())
        wg0, wo0 = wg1, wo1
    return s, o, reports


def delayed_steps(flux, mode, L, np_, P, dim, seed, dmax, steps):
    comm, k, _ = O.schedule(flux, mode, L, np_, P, dim, seed, dmax, 0, steps)
    return [n for n in range(steps) if not comm[n]]


@pytest.mark.parametrize("n", [32, 64])
def test_bench_at_config_two_cycles(n):
    # benchmark configuration on a smaller mesh: p=4, N_p=4 (5 levels), 8x8 subdomains,
    # CAA L=3 (cycle of 8: 5 communication + 3 delayed steps), CK4(5), CFL 0.1
    kw = dict(P=(8, 8), max_delay=3, flux="at", rk="ck45")
    s, o, rep = run_pair(2, (n, n), 4, 16, **kw)
    assert delayed_steps("at", "caa", 3, 4, (8, 8), 2, 0, 0, 16) == [5, 6, 7, 13, 14, 15]
    comm_g, k_g, _ = s.schedule(0, 16)
    comm_o, k_o, _ = O.schedule("at", "caa", 3, 4, (8, 8), 2, 0, 0, 0, 16)
    assert np.array_equal(comm_g, comm_o) and np.array_equal(k_g, k_o)
    s.close()


def test_bench_at_config_full_size_one_cycle():
    # the benchmarked workload itself: 256^2 quads, one whole schedule cycle (8 steps)
    kw = dict(P=(8, 8), max_delay=3, flux="at", rk="ck45")
    s, o, rep = run_pair(2, (256, 256), 4, 8, **kw)
    s.close()


@pytest.mark.parametrize("n", [4, 8])
def test_3d_tgv_at_config_ten_steps(n):
    # the 3D configuration on a smaller mesh: p=3, N_p=3 (4 levels), L=4 (cycle of 8:
    # 4 communication + 4 delayed steps), 2x2x2 subdomains, CK4(5), CFL 0.1
    kw = dict(P=(2, 2, 2), max_delay=4, flux="at", rk="ck45")
    s, o, rep = run_pair(3, (n, n, n), 3, 10, tgv=True, **kw)
    assert delayed_steps("at", "caa", 4, 3, (2, 2, 2), 3, 0, 0, 10) == [4, 5, 6, 7]
    s.close()


@pytest.mark.parametrize("flux", ["at", "std", "at_trace"])
def test_random_delay_p4(flux):
    # seeded random delays in {0, 1, 2} per subdomain interface and step, p=4
    kw = dict(P=(8, 8), max_delay=3, flux=flux, rk="ck45", delay_mode="random",
              random_delay_max=2, seed=20260301)
    s, o, rep = run_pair(2, (32, 32), 4, 12, **kw)
    comm_g, k_g, d_g = s.schedule(0, 12)
    comm_o, k_o, d_o = O.schedule(flux, "random", 3, 4, (8, 8), 2, 20260301, 2, 0, 12)
    assert np.array_equal(d_g, d_o) and np.array_equal(k_g, k_o)
    assert (d_o > 0).any()
    s.close()


def test_std_flux_p4_caa():
    kw = dict(P=(8, 8), max_delay=3, flux="std", rk="ck45")
    s, o, rep = run_pair(2, (32, 32), 4, 9, **kw)
    s.close()


@pytest.mark.parametrize("dim,n", [(2, 32), (3, 4)])
def test_df64_at_configs(dim, n):
    # the FP32-pair operator at the same configurations, held to the FP64 bounds
    if dim == 2:
        kw = dict(P=(8, 8), max_delay=3, flux="at", rk="ck45")
        run_pair(2, (n, n), 4, 16, precision="df64", **kw)[0].close()
    else:
        kw = dict(P=(2, 2, 2), max_delay=4, flux="at", rk="ck45")
        run_pair(3, (n, n, n), 3, 10, precision="df64", tgv=True, **kw)[0].close()


def test_increment_comparison_sees_a_wrong_weight_set():
    # The bound is tight enough to catch a plausible mistake on the delayed steps: the
    # oracle with a lower-order weight set (N_p = 2, three levels, Eq. 15 at r = 1) is far
    # outside it, the oracle with the right one (N_p = 4) inside.
    lo, hi = (-5.0, -5.0), (5.0, 5.0)
    u0, dt = cfl_dt(2, (32, 32), 4, lo, hi, False)
    kw = dict(n_elem=(32, 32), degree=4, P=(8, 8), max_delay=3, flux="at", rk="ck45", dt=dt)
    s = adg.Solver(**kw)
    right = O.Oracle(**kw)
    wrong = O.Oracle(at_np=2, **kw)
    for x in (s, right, wrong):
        x.set_state(u0)
        x.step(8)                     # one cycle of the N_p = 4 schedule
    wg = s.get_state()
    d_g, d_r, d_w = wg - u0, right.get_state() - u0, wrong.get_state() - u0
    good = np.linalg.norm(d_g - d_r) / np.linalg.norm(d_r)
    bad = np.linalg.norm(d_g - d_w) / np.linalg.norm(d_w)
    assert good < 1e-10, good
    assert bad > 1e3 * max(good, 1e-12), (good, bad)
    s.close()
