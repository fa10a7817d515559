"""Pins of the oracle's Taylor-Green initial condition and of its CFL time-step rule.

Neither is printed in the paper (the 3D configuration's initial condition and the rule
that turns a CFL number into a time step are builder-defined readings), so they are pinned
by what mathematics fixes about them rather than by retyping their formulas:

Taylor-Green vortex on [0, 2 pi]^3 (rho0 = V0 = 1, p0 = 1 / (gamma M^2)):
  * the z velocity is zero at every node;
  * the temperature is uniform: p / rho = p0 at every node, so the sound speed is 1/M and
    the flow Mach number is M;
  * domain means, worked by hand over a period: <rho> = 1, <rho u> = 0, <p> = p0,
    <rho |u|^2 / 2> = 1/8 (the density perturbation is orthogonal to |u|^2: the product's
    mean vanishes), and the pressure variance <(p - p0)^2> = 9/512;
  * the velocity field is divergence free: the discrete divergence at the nodes (nodal
    derivative of the degree-p interpolant) tends to zero at order p under refinement,
    where a wrong sign of one velocity component would leave it O(1);
  * the Gauss-quadrature means converge to those values under refinement.

CFL rule (reading O-7): dt = sigma h_min / ((2p + 1) max(|u| + c)), then shortened to
t_end / ceil(t_end / dt): checked on uniform states against values worked by hand, on a
state where a single node sets the maximum, on non-square elements (h_min), and for the
t_end rounding.
"""
import math

import numpy as np
import pytest

import oracle as O

GAMMA = 1.4


def tgv(n, p, mach=0.1):
    o = O.Oracle(dim=3, n_elem=(n, n, n), degree=p, lo=(0, 0, 0), hi=(2 * math.pi,) * 3, dt=1.0)
    return o, o.init_tgv(mach)


def quad_mean(o, n, p, f):
    """Domain mean of a nodal field f[elem][node] by the element Gauss rule."""
    x, w = O.gauss(p + 1)
    w3 = np.einsum("i,j,k->kji", w, w, w).reshape(-1)  # node index: xi_x fastest
    J = (math.pi / n) ** 3                                # (h/2)^3, h = 2 pi / n
    return float((f * w3[None, :]).sum() * J / (2 * math.pi) ** 3)


def primitives(u):
    rho = u[0]
    vel = u[1:4] / rho
    kin = 0.5 * (u[1] * vel[0] + u[2] * vel[1] + u[3] * vel[2])
    p = (GAMMA - 1.0) * (u[4] - kin)
    return rho, vel, kin, p


@pytest.mark.parametrize("mach", [0.1, 0.3])
def test_tgv_pointwise_invariants(mach):
    o, u = tgv(4, 3, mach)
    rho, vel, kin, p = primitives(u)
    p0 = 1.0 / (GAMMA * mach * mach)
    assert np.array_equal(u[3], np.zeros_like(u[3]))          # rho w = 0 exactly
    np.testing.assert_allclose(p / rho, p0, rtol=1e-13)       # uniform temperature
    c = np.sqrt(GAMMA * p / rho)
    np.testing.assert_allclose(c, 1.0 / mach, rtol=1e-13)     # Mach number M for V0 = 1
    assert np.abs(vel[0]).max() <= 1.0 and np.abs(vel[1]).max() <= 1.0


def test_tgv_domain_means_converge_to_closed_forms():
    p0 = 1.0 / (GAMMA * 0.01)
    errs = []
    for n in (2, 4, 8):
        o, u = tgv(n, 3)
        rho, vel, kin, p = primitives(u)
        m = {"rho": quad_mean(o, n, 3, rho) - 1.0,
             "mom": max(abs(quad_mean(o, n, 3, u[1 + d])) for d in range(3)),
             "p": quad_mean(o, n, 3, p) - p0,
             "kin": quad_mean(o, n, 3, kin) - 1.0 / 8.0,
             "pvar": quad_mean(o, n, 3, (p - p0) ** 2) - 9.0 / 512.0}
        errs.append(m)
    last = errs[-1]
    assert abs(last["rho"]) < 1e-12 and last["mom"] < 1e-12
    assert abs(last["p"]) < 1e-10 * p0
    assert abs(last["kin"]) < 1e-7 and abs(last["pvar"]) < 1e-7
    # the quadrature errors fall under refinement (spectral for these trigonometric fields)
    for key in ("kin", "pvar"):
        assert abs(errs[1][key]) < 0.1 * abs(errs[0][key]) + 1e-14
        assert abs(errs[2][key]) < 0.1 * abs(errs[1][key]) + 1e-14


def _divergence_max(n, p):
    o, u = tgv(n, p)
    rho, vel, _, _ = primitives(u)
    N = p + 1
    x, _ = O.gauss(N)
    D = np.array([[O.lagrange_deriv(x, a, x[i]) for a in range(N)] for i in range(N)])
    h = 2 * math.pi / n
    # nodes [elem][iz][iy][ix]
    vx = vel[0].reshape(-1, N, N, N)
    vy = vel[1].reshape(-1, N, N, N)
    dvx = np.einsum("ia,ezya->ezyi", D, vx) * (2.0 / h)
    dvy = np.einsum("ia,ezax->ezix", D, vy) * (2.0 / h)
    return np.abs(dvx + dvy).max()


def test_tgv_velocity_divergence_free():
    d = [_divergence_max(n, 3) for n in (2, 4, 8)]
    assert d[2] < 5e-3
    assert d[1] < 0.2 * d[0] and d[2] < 0.2 * d[1]


def _uniform(o, rho, vel, p):
    u = np.zeros(o.shape)
    u[0] = rho
    for d, v in enumerate(vel):
        u[1 + d] = rho * v
    u[-1] = p / (GAMMA - 1.0) + 0.5 * rho * sum(v * v for v in vel)
    return u


def test_dt_uniform_state_by_hand():
    # rho = 1, u = (0.5, 0.2), p = 1: |u| + c = sqrt(0.29) + sqrt(1.4) = 0.5385165 + 1.1832160 = 1.7217325
    # h = 10/16 = 0.625, p = 2: dt = 0.1 * 0.625 / (5 * 1.7217325) = 7.260129e-3
    o = O.Oracle(n_elem=(16, 16), degree=2, dt=1.0)
    u = _uniform(o, 1.0, (0.5, 0.2), 1.0)
    speed = math.sqrt(0.29) + math.sqrt(1.4)
    assert abs(speed - 1.7217325) < 1e-7
    dt = o.dt_from_cfl(u, 0.1, 0.0)
    assert abs(dt - 0.1 * 0.625 / (5 * speed)) < 1e-15
    assert abs(dt - 7.260129e-3) < 1e-9


def test_dt_non_square_elements_and_3d():
    # h = (10/20, 6/4) -> h_min = 0.5; rho = 2, at rest, p = 0.7: c = sqrt(1.4 * 0.35) = 0.7
    o = O.Oracle(n_elem=(20, 4), lo=(0.0, 0.0), hi=(10.0, 6.0), degree=3, dt=1.0)
    u = _uniform(o, 2.0, (0.0, 0.0), 0.7)
    assert abs(o.dt_from_cfl(u, 0.3, 0.0) - 0.3 * 0.5 / (7 * 0.7)) < 1e-15
    # 3D, h = 2 pi / 8, rho = 1, u = (0, 0, 1), p = 1/1.4 (c = 1): dt = 0.2 h / (3 * 2)
    o3 = O.Oracle(dim=3, n_elem=(8, 8, 8), lo=(0, 0, 0), hi=(2 * math.pi,) * 3, degree=1, dt=1.0)
    u3 = _uniform(o3, 1.0, (0.0, 0.0, 1.0), 1.0 / 1.4)
    assert abs(o3.dt_from_cfl(u3, 0.2, 0.0) - 0.2 * (2 * math.pi / 8) / 6.0) < 1e-15


def test_dt_maximum_taken_over_nodes():
    o = O.Oracle(n_elem=(8, 8), degree=2, dt=1.0)
    u = _uniform(o, 1.0, (0.0, 0.0), 1.0)
    base = o.dt_from_cfl(u, 0.1, 0.0)
    u[1, 37, 4] = 3.0                 # one node moving at u = 3
    u[-1, 37, 4] += 0.5 * 9.0
    fast = o.dt_from_cfl(u, 0.1, 0.0)
    assert abs(fast - 0.1 * 1.25 / (5 * (3.0 + math.sqrt(1.4)))) < 1e-15
    assert fast < base


def test_dt_rounding_to_t_end():
    o = O.Oracle(n_elem=(16, 16), degree=2, dt=1.0)
    u = _uniform(o, 1.0, (0.5, 0.2), 1.0)
    raw = o.dt_from_cfl(u, 0.1, 0.0)                 # 7.2601e-3: 1 / raw = 137.74
    dt = o.dt_from_cfl(u, 0.1, 1.0)
    assert abs(dt - 1.0 / 138) < 1e-17 and dt <= raw
    # t_end an exact multiple: unchanged up to rounding
    dt2 = o.dt_from_cfl(u, 0.1, 50 * raw)
    assert abs(dt2 - raw) < 1e-15
