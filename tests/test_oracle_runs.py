"""Pins of full oracle runs: conservation in every flux mode, the zero-delay special cases
equal the synchronous algorithm bit for bit, free-stream preservation under delays, the
delay-error orders the paper reports (first order with the standard flux, N_p+1 with AT),
and spatial convergence of the synchronous scheme."""
import numpy as np
import pytest

import oracle as O
from paper_2603_28710_gb300.inputs import random_state


def vortex_run(flux, n=8, p=2, P=(2, 2), L=2, rk="ck45", steps=12, dt=0.01, **kw):
    o = O.Oracle(n_elem=(n, n), degree=p, P=P, max_delay=L, flux=flux, rk=rk, dt=dt, **kw)
    u0 = o.init_vortex()
    o.set_state(u0)
    o.step(steps)
    return o, u0, o.get_state()


@pytest.mark.parametrize("flux,mode", [("sync", "caa"), ("std", "caa"), ("at", "caa"),
                                       ("at_trace", "caa"), ("std", "random"), ("at", "random"),
                                       ("at_trace", "random")])
def test_conservation_every_mode(flux, mode):
    o, u0, u1 = vortex_run(flux, delay_mode=mode, random_delay_max=2, seed=9, steps=15)
    s0, s1 = o.conservation(u0), o.conservation(u1)
    assert np.abs(s1 - s0).max() < 1e-13 * np.abs(s0).max()
    assert np.abs(u1 - u0).max() > 1e-3  # the state did move


@pytest.mark.parametrize("flux,kw", [("at", dict(P=(1, 1), L=3)), ("std", dict(P=(1, 1), L=3)),
                                     ("at", dict(L=0)), ("std", dict(L=1)),
                                     ("at", dict(delay_mode="random", random_delay_max=0))])
def test_zero_delay_cases_equal_synchronous_bitwise(flux, kw):
    _, _, ref = vortex_run("sync", steps=7)
    _, _, got = vortex_run(flux, steps=7, **kw)
    assert np.array_equal(ref, got)


def test_delayed_runs_differ_from_synchronous():
    _, _, ref = vortex_run("sync", steps=8)
    for flux in ("std", "at", "at_trace"):
        _, _, got = vortex_run(flux, steps=8, L=3)
        assert np.abs(got - ref).max() > 1e-9


@pytest.mark.parametrize("flux", ["std", "at", "at_trace"])
def test_free_stream_preserved_under_delay(flux):
    o = O.Oracle(n_elem=(8, 8), degree=2, P=(2, 2), max_delay=3, flux=flux, rk="rk33", dt=0.01)
    u = np.zeros(o.shape)
    for v, val in enumerate([1.1, 0.3, -0.2, 3.0]):
        u[v] = val
    o.set_state(u)
    o.step(14)
    assert np.abs(o.get_state() - u).max() < 1e-13


def _delay_error_slopes(p, rk, n, T, base, levels=3, **kw):
    res = {}
    for flux in ("sync", "std", "at", "at_trace"):
        out = []
        for j in range(levels):
            nsteps = int(round(T / base)) * 2 ** j
            o = O.Oracle(n_elem=(n, n), degree=p, P=(4, 4), max_delay=4, flux=flux, rk=rk,
                         dt=T / nsteps, **kw)
            o.set_state(o.init_vortex())
            o.step(nsteps)
            out.append(o.get_state())
        res[flux] = out
    slopes = {}
    for flux in ("std", "at", "at_trace"):
        d = np.array([np.linalg.norm(res[flux][j] - res["sync"][j]) for j in range(levels)])
        slopes[flux] = np.log2(d[:-1] / d[1:])
    return slopes


def test_delay_error_orders_np1():
    # ADG(1)-LSERK2 vs ADG(1)-AT2-LSERK2: delay error O(dt) with the standard flux,
    # O(dt^2) with the AT flux (Section 5.3, Fig. 6 claims)
    s = _delay_error_slopes(1, "rk22", 16, 0.5, 0.01, levels=4)
    assert np.all(np.abs(s["std"] - 1.0) < 0.15), s
    assert np.all(np.abs(s["at"] - 2.0) < 0.15), s
    assert np.all(np.abs(s["at_trace"] - 2.0) < 0.15), s


def test_delay_error_orders_np2():
    # ADG(2)-LSERK3 vs ADG(2)-AT3-LSERK3: O(dt) vs O(dt^3) (Fig. 7 claims)
    s = _delay_error_slopes(2, "rk33", 8, 0.4, 0.01, levels=3)
    assert np.all(np.abs(s["std"] - 1.0) < 0.15), s
    assert np.all(np.abs(s["at"] - 3.0) < 0.2), s


def test_delay_error_orders_random_mode():
    # seeded per-interface delays in {0,1,2}: same orders as the fixed schedule
    s = _delay_error_slopes(1, "rk22", 16, 0.5, 0.01, levels=3, delay_mode="random",
                            random_delay_max=2, seed=20260301)
    assert np.all(np.abs(s["std"] - 1.0) < 0.2), s
    assert np.all(np.abs(s["at"] - 2.0) < 0.2), s


def test_synchronous_spatial_convergence():
    errs = []
    for n in (8, 16, 32):
        o0 = O.Oracle(n_elem=(n, n), degree=2, rk="ck45", dt=1.0)
        u0 = o0.init_vortex()
        dt = o0.dt_from_cfl(u0, 0.2, 0.5)
        o = O.Oracle(n_elem=(n, n), degree=2, rk="ck45", dt=dt)
        o.set_state(u0)
        o.step(int(round(0.5 / dt)))
        errs.append(o.l2_error_vortex(o.get_state(), 0.5))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates[-1] > 2.5), rates


def test_3d_tgv_mirror_symmetry_and_conservation():
    n, p = 4, 2
    o = O.Oracle(dim=3, n_elem=(n, n, n), lo=(0, 0, 0), hi=(2 * np.pi,) * 3, degree=p, P=(2, 2, 2),
                 max_delay=2, flux="at", rk="rk33", dt=0.01)
    u0 = o.init_tgv(0.1)
    o.set_state(u0)
    o.step(6)
    u = o.get_state()
    assert np.abs(o.conservation(u) - o.conservation(u0)).max() < 1e-12 * np.abs(o.conservation(u0)).max()
    nn = p + 1
    r = u.reshape(5, n, n, n, nn, nn, nn)          # var, ez, ey, ex, c, b, a
    m = r[:, ::-1, :, :, ::-1, :, :]                 # z -> 2 pi - z
    sign = np.array([1, 1, 1, -1, 1]).reshape(5, 1, 1, 1, 1, 1, 1)
    np.testing.assert_allclose(m * sign, r, rtol=0, atol=1e-12)
    assert np.abs(u[3]).max() > 1e-6   # z-momentum developed


def test_random_state_run_is_finite_and_conservative():
    o = O.Oracle(n_elem=(6, 6), degree=3, P=(3, 2), max_delay=2, flux="at", rk="rk33", dt=2e-4)
    u0 = random_state(o.shape, 2, seed=21)
    o.set_state(u0)
    o.step(5)
    u = o.get_state()
    assert np.isfinite(u).all()
    assert np.abs(o.conservation(u) - o.conservation(u0)).max() < 1e-13


def test_all_cores_build_equals_single_threaded_bitwise():
    # the OpenMP variant (timing only) splits elements over threads; each element's
    # arithmetic is unchanged, so runs and residuals agree bit for bit
    kw = dict(n_elem=(16, 16), degree=3, P=(4, 4), max_delay=3, flux="at", rk="ck45", dt=2e-3)
    a, b = O.Oracle(**kw), O.Oracle(parallel=True, **kw)
    u0 = a.init_vortex()
    for o in (a, b):
        o.set_state(u0)
        o.step(9)
    assert np.array_equal(a.get_state(), b.get_state())
    assert np.array_equal(a.rhs(u0), b.rhs(u0))
    assert O.threads(False) == 1 and O.threads(True) >= 1
