"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, value by value.

Tolerances (FP64 operator): operator output and each step within 1e-12 relative L2 (the
oracle sums its dense quadrature in a different order, so results agree to rounding, not
bit for bit); 1e-10 after a full run; integer schedule data bit for bit.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_28710_gb300 import adg
from paper_2603_28710_gb300.inputs import random_state

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-12
RUN_TOL = 1e-10


def summand_scale(u_el, dim, degree, h, gamma=1.4):
    """Per (element, variable) size of the terms the operator sums at one node:
    S = sum_d (2/h_d) Lambda max_nodes |F_d(w)|, Lambda = max_i (sum_a |w_a l_i'(x_a) / w_i|
    + |l_i(1) / w_i| + |l_i(-1) / w_i|) on the reference element.  The weak derivative
    cancels terms of this size, so an FP64 evaluation in any summation order is exact to a
    small multiple of eps * S at each node, whatever the (possibly tiny) result."""
    n = degree + 1
    x, w = O.gauss(n)
    lam = max(sum(abs(w[a] * O.lagrange_deriv(x, i, x[a]) / w[i]) for a in range(n))
              + abs(O.lagrange(x, i, 1.0) / w[i]) + abs(O.lagrange(x, i, -1.0) / w[i])
              for i in range(n))
    ne, nv, nd = u_el.shape
    S = np.zeros((ne, nv))
    for e in range(ne):
        for d in range(dim):
            F = np.array([O.euler_flux(dim, gamma, u_el[e, :, q], d) for q in range(nd)])
            S[e] += (2.0 / h[d]) * lam * np.abs(F).max(axis=0)
    return S


def elementwise_ok(kg, ko, S):
    """|kg - ko| <= 1e-12 max|ko| + 256 eps S at every node (kg, ko: [elem][var][node]).
    256: each side's node value sums about 2d (p+1) + 2d products of this size, each side
    rounds them in its own order, and the face terms carry the rounding of the traces they
    are evaluated from (measured on GB300: up to about 120 eps S on the 3D Taylor-Green
    vortex)."""
    bound = 1e-12 * np.abs(ko).max() + 256 * 2.0 ** -53 * S[:, :, None]
    excess = (np.abs(kg - ko) / bound).max()
    return excess <= 1.0, excess


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_28710_gb300 import build
    build.build()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def pair(dim=2, n_elem=(8, 8), degree=2, lo=None, hi=None, **kw):
    lo = lo or (-5.0,) * dim
    hi = hi or (5.0,) * dim
    s = adg.Solver(dim=dim, n_elem=n_elem, degree=degree, lo=lo, hi=hi, **kw)
    okw = {k: v for k, v in kw.items() if k in ("P", "max_delay", "flux", "rk", "delay_mode",
                                                 "random_delay_max", "at_np", "seed", "gamma", "dt")}
    o = O.Oracle(dim=dim, n_elem=n_elem, degree=degree, lo=lo, hi=hi, **okw)
    return s, o


# ---- operator ------------------------------------------------------------------------

RHS_CASES = [(2, (5, 3), p) for p in range(1, 8)] + [(3, (3, 2, 2), p) for p in range(1, 6)] + \
            [(2, (1, 4), 2), (3, (1, 1, 2), 2), (2, (16, 9), 4)]


@pytest.mark.parametrize("dim,n_elem,p", RHS_CASES)
def test_rhs_random_state(dim, n_elem, p):
    lo = (-5.0, -2.0, 0.0)[:dim]
    hi = (5.0, 3.0, 1.5)[:dim]            # non-square elements
    s, o = pair(dim, n_elem, p, lo=lo, hi=hi, dt=1e-3)
    u = random_state(s.shape, dim, seed=100 + p)
    kg, ko = s.rhs(u), o.rhs(u)
    assert rel(kg, ko) < STEP_TOL
    assert np.abs(kg - ko).max() < 1e-11 * np.abs(ko).max()


@pytest.mark.parametrize("p", [2, 4])
def test_rhs_vortex_device_buffers(p):
    import torch
    s, o = pair(2, (12, 12), p, dt=1e-3)
    u = o.init_vortex()
    ud = torch.from_numpy(u).cuda()
    kd = torch.empty_like(ud)
    s.rhs(ud, kd)
    assert rel(kd.cpu().numpy(), o.rhs(u)) < STEP_TOL


# ---- stepping: every flux mode, delay mode and RK scheme -----------------------------

MODES = [("sync", "caa", 1), ("std", "caa", 3), ("at", "caa", 2), ("at_trace", "caa", 2),
         ("std", "random", 0), ("at", "random", 0), ("at_trace", "random", 0)]


@pytest.mark.parametrize("flux,mode,L", MODES)
@pytest.mark.parametrize("rk", ["rk22", "rk33", "ck45"])
def test_steps_match_oracle(flux, mode, L, rk):
    kw = dict(P=(2, 3), max_delay=L, flux=flux, rk=rk, delay_mode=mode, random_delay_max=2,
              seed=20260301, dt=0.01)
    s, o = pair(2, (8, 9), 2, **kw)
    u0 = o.init_vortex(beta=3.0, x0=0.7, y0=-0.4)
    s.set_state(u0)
    o.set_state(u0)
    for n in range(12):
        s.step(1)
        o.step(1)
        assert rel(s.get_state(), o.get_state()) < STEP_TOL, f"step {n}"
    comm_g, k_g, d_g = s.schedule(0, 12)
    comm_o, k_o, d_o = O.schedule(flux, mode, L, 2, (2, 3), 2, 20260301, 2, 0, 12)
    assert np.array_equal(comm_g, comm_o) and np.array_equal(k_g, k_o) and np.array_equal(d_g, d_o)


@pytest.mark.parametrize("flux", ["std", "at", "at_trace"])
def test_3d_steps_match_oracle(flux):
    kw = dict(P=(2, 2, 2), max_delay=2, flux=flux, rk="rk33", dt=0.01)
    s, o = pair(3, (4, 4, 4), 2, lo=(0, 0, 0), hi=(2 * np.pi,) * 3, **kw)
    u0 = o.init_tgv(0.1)
    s.set_state(u0)
    o.set_state(u0)
    for n in range(7):
        s.step(1)
        o.step(1)
        assert rel(s.get_state(), o.get_state()) < STEP_TOL, f"step {n}"


def test_full_run_small_vortex_config():
    # 16^2 quads, p=2, 2x2 subdomains, L=2, AT flux, CK4(5), CFL 0.1 to t_end = 1
    o0 = O.Oracle(n_elem=(16, 16), degree=2, dt=1.0)
    u0 = o0.init_vortex()
    dt = o0.dt_from_cfl(u0, 0.1, 1.0)
    kw = dict(P=(2, 2), max_delay=2, flux="at", rk="ck45", dt=dt)
    s, o = pair(2, (16, 16), 2, **kw)
    s.set_state(u0)
    o.set_state(u0)
    nsteps = int(round(1.0 / dt))
    s.step(nsteps)
    o.step(nsteps)
    assert rel(s.get_state(), o.get_state()) < RUN_TOL
    # the library's own CFL time step agrees with the oracle's (without the rounding to
    # t_end, whose ceil() can flip on a one-ulp difference)
    s2 = adg.Solver(n_elem=(16, 16), degree=2, cfl=0.1)
    s2.set_state(u0)
    dt_raw = o0.dt_from_cfl(u0, 0.1, 0.0)
    assert abs(s2.info()["dt"] - dt_raw) < 1e-14 * dt_raw


# ---- full-size workloads (sampled / single step) ---------------------------------------

def test_large_vortex_rhs_sampled():
    # 256^2 quads, p=4: operator at sampled elements, including subdomain-boundary ones,
    # compared node by node
    s = adg.Solver(n_elem=(256, 256), degree=4, P=(8, 8), max_delay=3, flux="at", dt=1e-4)
    o = O.Oracle(n_elem=(256, 256), degree=4, dt=1e-4)
    u = o.init_vortex()
    k = s.rhs(u)
    rng = np.random.default_rng(0)
    sel = np.concatenate([[0, 31, 32, 255, 256 * 31 + 31, 65535], rng.integers(0, 65536, 200)])
    ko = o.rhs_elements(u, sel)
    kg = k[:, sel].transpose(1, 0, 2)
    S = summand_scale(u[:, sel].transpose(1, 0, 2), 2, 4, (10 / 256, 10 / 256))
    ok, excess = elementwise_ok(kg, ko, S)
    assert ok, excess


def test_large_vortex_one_step_full_compare():
    # the benchmarked configuration: 256^2, p=4, 8x8 subdomains, CAA L=3, AT, CK4(5)
    kw = dict(P=(8, 8), max_delay=3, flux="at", rk="ck45", dt=1.2e-4)
    s, o = pair(2, (256, 256), 4, **kw)
    u0 = o.init_vortex()
    s.set_state(u0)
    o.set_state(u0)
    s.step(1)
    o.step(1)
    assert rel(s.get_state(), o.get_state()) < STEP_TOL


def test_large_tgv_rhs_sampled():
    # 64^3 hexes, p=3 (Taylor-Green), sampled elements
    s = adg.Solver(dim=3, n_elem=(64, 64, 64), degree=3, lo=(0, 0, 0), hi=(2 * np.pi,) * 3,
                   P=(8, 8, 8), max_delay=4, flux="at", dt=1e-3)
    o = O.Oracle(dim=3, n_elem=(64, 64, 64), degree=3, lo=(0, 0, 0), hi=(2 * np.pi,) * 3, dt=1e-3)
    s.init_tgv(0.1)
    u = s.get_state()
    uo = o.init_tgv(0.1)
    assert rel(u, uo) < 1e-14
    k = s.rhs(uo)
    rng = np.random.default_rng(1)
    sel = np.concatenate([[0, 7, 8, 64 * 64 * 64 - 1], rng.integers(0, 64 ** 3, 60)])
    kg, ko = k[:, sel].transpose(1, 0, 2), o.rhs_elements(uo, sel)
    S = summand_scale(uo[:, sel].transpose(1, 0, 2), 3, 3, (2 * np.pi / 64,) * 3)
    ok, excess = elementwise_ok(kg, ko, S)
    assert ok, excess


# ---- invariants and diagnostics -------------------------------------------------------

@pytest.mark.parametrize("flux,mode", [("sync", "caa"), ("std", "caa"), ("at", "caa"),
                                       ("at_trace", "caa"), ("at", "random")])
def test_conservation_on_gpu(flux, mode):
    s = adg.Solver(n_elem=(32, 32), degree=3, P=(4, 4), max_delay=3, flux=flux, delay_mode=mode,
                   random_delay_max=2, seed=5, dt=2e-3)
    s.init_vortex()
    c0 = s.conservation()
    s.step(40)
    c1 = s.conservation()
    assert np.abs(c1 - c0).max() < 1e-12 * np.abs(c0).max()


def test_diagnostics_match_oracle():
    s, o = pair(2, (10, 10), 3, dt=1e-3)
    s.init_vortex(t=0.3, beta=4.0, x0=0.5, y0=1.0)
    uo = o.init_vortex(t=0.3, beta=4.0, x0=0.5, y0=1.0)
    assert rel(s.get_state(), uo) < 1e-14
    scale = o.conservation(np.abs(uo)).max()      # size of the summands
    np.testing.assert_allclose(s.conservation(), o.conservation(uo), rtol=1e-13, atol=1e-14 * scale)
    np.testing.assert_allclose(s.l2_error_vortex(0.0), o.l2_error_vortex(uo, 0.0), rtol=1e-11)
    assert s.check_finite()


def test_zero_delay_equals_sync_on_gpu():
    ref = adg.Solver(n_elem=(8, 8), degree=2, flux="sync", dt=0.01)
    at0 = adg.Solver(n_elem=(8, 8), degree=2, P=(2, 2), flux="at", max_delay=0, dt=0.01)
    p1 = adg.Solver(n_elem=(8, 8), degree=2, P=(1, 1), flux="std", max_delay=3, dt=0.01)
    for s in (ref, at0, p1):
        s.init_vortex()
        s.step(9)
    assert np.array_equal(ref.get_state(), at0.get_state())
    assert np.array_equal(ref.get_state(), p1.get_state())


def test_errors_and_edge_cases():
    s = adg.Solver(n_elem=(4, 4), degree=1, dt=0.01)
    with pytest.raises(adg.AdgError) as e:
        s.step(1)
    assert e.value.status == 7
    with pytest.raises(adg.AdgError):
        s.set_state(np.zeros(5))
    with pytest.raises(adg.AdgError):
        adg.Solver(n_elem=(6, 6), P=(4, 4), flux="at")
    with pytest.raises(adg.AdgError):
        adg.Solver(dim=3, n_elem=(2, 2, 2), degree=6)
    s.init_vortex()
    u = s.get_state()
    s.step(0)
    assert np.array_equal(s.get_state(), u)
    u[0, 0, 0] = np.nan
    bad = adg.Solver(n_elem=(4, 4), degree=1, dt=0.01)
    bad.set_state(u)
    assert not bad.check_finite()
