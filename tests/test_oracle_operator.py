"""Pins of the oracle's DG operator M^{-1} L_h (Eq. 6-7): free-stream preservation,
discrete conservation, consistency with the exact vortex, symmetries, and 3D vs 2D."""
import numpy as np
import pytest

import oracle as O
from paper_2603_28710_gb300.inputs import random_state

G = 1.4


def mk(dim=2, n=8, p=2, **kw):
    if dim == 2:
        return O.Oracle(dim=2, n_elem=(n, n), lo=(-5, -5), hi=(5, 5), degree=p, **kw)
    return O.Oracle(dim=3, n_elem=(n, n, n), lo=(0, 0, 0), hi=(2 * np.pi,) * 3, degree=p, **kw)


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (2, 4), (3, 1), (3, 3)])
def test_free_stream_preserved(dim, p):
    o = mk(dim, 4, p)
    u = np.zeros(o.shape)
    state = [1.3, 0.4, -0.7, 0.2, 5.1][:dim + 1] + [5.1]
    for v in range(o.nv):
        u[v] = state[v]
    k = o.rhs(u)
    assert np.abs(k).max() < 1e-12


@pytest.mark.parametrize("dim,p", [(2, 2), (2, 3), (3, 2)])
def test_rhs_is_conservative(dim, p):
    o = mk(dim, 4, p)
    u = random_state(o.shape, dim, seed=5)
    k = o.rhs(u)
    s = o.conservation(k)
    scale = np.abs(k).max() * 100
    assert np.abs(s).max() < 1e-13 * scale


def _exact_dwdt(o, delta=1e-4):
    # time derivative of the exact (translating) vortex, by a 4th-order central difference
    f = lambda t: o.init_vortex(t=t)
    return (-f(2 * delta) + 8 * f(delta) - 8 * f(-delta) + f(-2 * delta)) / (12 * delta)


@pytest.mark.parametrize("p", [2, 3])
def test_rhs_consistent_with_exact_vortex(p):
    errs = []
    for n in (8, 16, 32):
        o = mk(2, n, p)
        u = o.init_vortex()
        d = o.rhs(u) - _exact_dwdt(o)
        errs.append(np.sqrt(o.conservation(d * d).sum()))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < errs[0] / 8
    assert np.all(rates > p - 0.6), rates


def test_transpose_symmetry_2d():
    # swapping x and y (elements, nodes, momentum components) commutes with the operator
    o = mk(2, 6, 3)
    u = random_state(o.shape, 2, seed=11)
    n, nn = 6, 4

    def tr(a):
        a = a.reshape(4, n, n, nn, nn)            # var, ey, ex, b, a
        a = a.transpose(0, 2, 1, 4, 3)[[0, 2, 1, 3]]
        return a.reshape(4, n * n, nn * nn)

    np.testing.assert_allclose(o.rhs(tr(u)), tr(o.rhs(u)), rtol=0, atol=1e-12)


def test_shift_equivariance():
    o = mk(2, 6, 2)
    u = random_state(o.shape, 2, seed=12)

    def shift(a):
        return np.roll(a.reshape(4, 6, 6, 9), 1, axis=2).reshape(4, 36, 9)

    np.testing.assert_allclose(o.rhs(shift(u)), shift(o.rhs(u)), rtol=0, atol=0)


def test_3d_extruded_vortex_matches_2d():
    n, p = 6, 2
    o2 = O.Oracle(dim=2, n_elem=(n, n), lo=(-5, -5), hi=(5, 5), degree=p)
    o3 = O.Oracle(dim=3, n_elem=(n, n, 2), lo=(-5, -5, 0), hi=(5, 5, 1), degree=p)
    u2, u3 = o2.init_vortex(), o3.init_vortex()
    nn = p + 1
    u3r = u3.reshape(5, 2, n, n, nn, nn, nn)    # var, ez, ey, ex, c, b, a
    for ez in range(2):
        for c in range(nn):
            np.testing.assert_array_equal(u3r[[0, 1, 2, 4], ez, :, :, c].reshape(4, n * n, nn * nn), u2)
    k2, k3 = o2.rhs(u2), o3.rhs(u3).reshape(5, 2, n, n, nn, nn, nn)
    for ez in range(2):
        for c in range(nn):
            np.testing.assert_allclose(k3[[0, 1, 2, 4], ez, :, :, c].reshape(4, n * n, nn * nn), k2,
                                       rtol=0, atol=1e-11)
    assert np.abs(k3[3]).max() < 1e-11


def test_rhs_elements_matches_full_rhs():
    o = mk(2, 6, 2)
    u = random_state(o.shape, 2, seed=13)
    k = o.rhs(u)
    sel = np.array([0, 5, 17, 35])
    np.testing.assert_array_equal(o.rhs_elements(u, sel), k[:, sel].transpose(1, 0, 2))


def test_l2_error_of_interpolant_converges():
    errs = []
    for n in (8, 16, 32):
        o = mk(2, n, 2)
        errs.append(o.l2_error_vortex(o.init_vortex(), 0.0))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates > 2.6), rates   # interpolation error O(h^{p+1})
