"""Pins of the oracle's Euler flux (Eq. 2-3), Rusanov flux (Eq. 8-9) and schedules
(Algorithms 2 and 3, seeded random-delay mode)."""
import math

import numpy as np
import pytest

import oracle as O
from conftest import golden

G = 1.4


def test_euler_flux_hand_cases():
    for row in golden("euler_flux_cases.txt"):
        d = int(row[1])
        w = [float(v) for v in row[2:6]]
        ref = [float(v) for v in row[6:10]]
        np.testing.assert_allclose(O.euler_flux(2, G, w, d), ref, rtol=0, atol=1e-13)


def test_euler_flux_3d_reduces_to_2d():
    w2 = np.array([0.5, 1.0, -2.0, 7.0])
    w3 = np.array([0.5, 1.0, -2.0, 0.0, 7.0])
    for d in (0, 1):
        f2 = O.euler_flux(2, G, w2, d)
        f3 = O.euler_flux(3, G, w3, d)
        np.testing.assert_allclose(f3[[0, 1, 2, 4]], f2, atol=1e-14)
        assert f3[3] == 0.0
    # z-flux of a state with no z-velocity: only the pressure enters the z-momentum
    fz = O.euler_flux(3, G, w3, 2)
    np.testing.assert_allclose(fz, [0, 0, 0, 0.8, 0], atol=1e-14)


def test_llf_hand_case():
    # w- = (1,0,0,2.5): p=1, c^2=1.4; w+ = (1,0,0,5): p=2, c^2=2.8; n = +x
    # lambda = 1/2 max(sqrt(1.4), sqrt(2.8)) = sqrt(2.8)/2
    # F^.n = 1/2 (F(w-)+F(w+)).n + lambda/2 (w- - w+) = (0, 1.5, 0, -2.5 sqrt(2.8)/4)
    f = O.llf(2, G, [1, 0, 0, 2.5], [1, 0, 0, 5.0], [1.0, 0.0])
    np.testing.assert_allclose(f, [0, 1.5, 0, -2.5 * math.sqrt(2.8) / 4], rtol=0, atol=1e-15)


def test_llf_consistency_and_antisymmetry():
    rng = np.random.default_rng(3)
    for dim in (2, 3):
        for _ in range(50):
            a = np.concatenate([[rng.uniform(0.5, 2)], rng.uniform(-1, 1, dim), [rng.uniform(4, 6)]])
            b = np.concatenate([[rng.uniform(0.5, 2)], rng.uniform(-1, 1, dim), [rng.uniform(4, 6)]])
            for d in range(dim):
                n = np.zeros(dim)
                n[d] = 1.0
                np.testing.assert_allclose(O.llf(dim, G, a, a, n), O.euler_flux(dim, G, a, d),
                                           rtol=1e-15, atol=1e-15)
                # F^(a, b, n) == -F^(b, a, -n) bit for bit (conservation across a face)
                assert np.array_equal(O.llf(dim, G, a, b, n), -O.llf(dim, G, b, a, -n))


def test_splitmix64_reference_outputs():
    for row in golden("splitmix64.txt"):
        i, ref = int(row[0]), int(row[1], 16)
        assert O.splitmix64(i * 0x9E3779B97F4A7C15) == ref


@pytest.mark.parametrize("L", [1, 2, 3, 5])
def test_caa_std_schedule_closed_form(L):
    comm, k, _ = O.schedule("std", "caa", L, 2, (2, 2), 2, 0, 0, 0, 60)
    n = np.arange(60)
    assert np.array_equal(comm, (n % L == 0).astype(np.int32))
    assert np.array_equal(k, n % L)


@pytest.mark.parametrize("L,np_", [(0, 1), (1, 1), (2, 2), (3, 4), (4, 2), (10, 2)])
def test_caa_at_schedule_closed_form(L, np_):
    comm, k, _ = O.schedule("at", "caa", L, np_, (2, 2), 2, 0, 0, 0, 80)
    n = np.arange(80)
    cyc = L + np_ + 1
    assert np.array_equal(comm, (n % cyc < np_ + 1).astype(np.int32))
    ref_k = np.where(n % cyc < np_ + 1, 0, n % cyc - np_)
    assert np.array_equal(k, ref_k)
    # the first N_p+1 steps are communication steps (history warm-up)
    assert np.all(comm[:np_ + 1] == 1)
    # an offset window equals the same slice of a full run
    c2, k2, _ = O.schedule("at", "caa", L, np_, (2, 2), 2, 0, 0, 13, 20)
    assert np.array_equal(c2, comm[13:33]) and np.array_equal(k2, k[13:33])


def test_random_schedule_definition_and_fallback():
    P, dim, seed, dmax, np_ = (2, 3), 2, 20260301, 2, 2
    nif = O.num_interfaces(dim, P)
    assert nif == 12
    comm, k, dl = O.schedule("at", "random", 0, np_, P, dim, seed, dmax, 0, 50)
    for n in range(50):
        for f in range(nif):
            kt = O.splitmix64(seed ^ (n * nif + f)) % (dmax + 1)
            if n - kt - np_ < 0:
                kt = 0
            assert dl[n, f] == kt
        assert k[n] == dl[n].max() and comm[n] == int(dl[n].max() == 0)
    # delays are spread over 0..dmax
    assert set(np.unique(dl[10:])) == {0, 1, 2}
    # standard flux only needs level n-k to exist
    _, _, dls = O.schedule("std", "random", 0, np_, P, dim, seed, dmax, 0, 5)
    assert dls[1].max() <= 1 and dls[0].max() == 0


def test_num_interfaces():
    assert O.num_interfaces(2, (1, 1)) == 0
    assert O.num_interfaces(2, (8, 8)) == 128
    assert O.num_interfaces(2, (4, 1)) == 4
    assert O.num_interfaces(3, (8, 8, 8)) == 3 * 512
