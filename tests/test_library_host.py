"""CPU-side checks of the CUDA library: it loads, exports every declared symbol, and its
host logic (basis, AT weights, RK tables, schedules) agrees with the oracle.  No GPU."""
import re
import os

import numpy as np
import pytest

import oracle as O
from paper_2603_28710_gb300 import adg
from conftest import ROOT, golden


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2603_28710_gb300 import build
    build.build()


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "adg.h")).read()
    declared = set(re.findall(r"\b(adg_[a-z0-9_]+)\s*\(", hdr))
    assert declared == set(adg.SYMBOLS)
    L = adg.lib()
    for name in declared:
        assert hasattr(L, name), name


@pytest.mark.parametrize("n", range(1, 10))
def test_gauss_matches_oracle(n):
    x, w = adg.host_gauss(n)
    xo, wo = O.gauss(n)
    np.testing.assert_allclose(x, xo, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, wo, rtol=0, atol=2e-15)


@pytest.mark.parametrize("np_", range(0, 8))
def test_at_weights_match_oracle(np_):
    for km in (0.0, 0.14965902, 1.0, 2.632124764, 3.958, 7.0):
        c = adg.host_at_coeffs(np_, km)
        co = O.at_coeffs(np_, km)
        np.testing.assert_allclose(c, co, rtol=1e-12, atol=1e-12 * np.abs(co).max())


@pytest.mark.parametrize("scheme", ["rk22", "rk33", "ck45"])
def test_rk_tables_match_oracle(scheme):
    a, b, c = adg.host_rk(scheme)
    ao, bo, co, _, _ = O.rk_tableau(scheme)
    assert np.array_equal(b, bo)
    if scheme == "ck45":
        assert np.array_equal(a, ao)
    else:
        assert np.array_equal(a[:-1], ao[:-1])
    np.testing.assert_allclose(c, co, rtol=0, atol=1e-15)


SCHEDULES = [("sync", "caa", 1, 2), ("std", "caa", 1, 2), ("std", "caa", 3, 4), ("at", "caa", 0, 2),
             ("at", "caa", 2, 2), ("at", "caa", 3, 4), ("at_trace", "caa", 4, 3), ("at", "caa", 10, 2)]


@pytest.mark.parametrize("flux,mode,L,np_", SCHEDULES)
def test_caa_schedule_bit_exact(flux, mode, L, np_):
    for P, dim in (((2, 2), 2), ((8, 8), 2), ((2, 4, 2), 3)):
        a = adg.host_schedule(flux, mode, L, np_, P, dim, 0, 0, 0, 200)
        b = O.schedule(flux, mode, L, np_, P, dim, 0, 0, 0, 200)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
        a2 = adg.host_schedule(flux, mode, L, np_, P, dim, 0, 0, 137, 50)
        b2 = O.schedule(flux, mode, L, np_, P, dim, 0, 0, 137, 50)
        for x, y in zip(a2, b2):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("flux", ["sync", "std", "at", "at_trace"])
@pytest.mark.parametrize("dmax,seed", [(0, 1), (2, 20260301), (5, 7), (15, 2 ** 63 + 11)])
def test_random_schedule_bit_exact(flux, dmax, seed):
    for P, dim in (((8, 8), 2), ((2, 1), 2), ((2, 2, 2), 3)):
        a = adg.host_schedule(flux, "random", 0, 3, P, dim, seed, dmax, 0, 120)
        b = O.schedule(flux, "random", 0, 3, P, dim, seed, dmax, 0, 120)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_num_interfaces_match():
    for dim, P in ((2, (1, 1)), (2, (8, 8)), (2, (4, 1)), (3, (8, 8, 8)), (3, (1, 2, 1))):
        assert adg.host_num_interfaces(dim, P) == O.num_interfaces(dim, P)


def test_dof_count_matches_table3():
    # DoFs = nodes x variables (Table 3): N_E (N_p+1)^d (d+2) with N_p = 2
    for row in golden("dof_table3.txt"):
        dim, ne, dofs, tol = int(row[0]), int(row[2]), int(row[3]), int(row[4])
        assert abs(ne * 3 ** dim * (dim + 2) - dofs) <= tol


def test_bad_arguments_rejected_without_gpu():
    with pytest.raises(adg.AdgError):
        adg.host_gauss(0)
    with pytest.raises(adg.AdgError):
        adg.host_at_coeffs(9, 1.0)
    # the bounded-wait probe checks its limit before any device work
    with pytest.raises(adg.AdgError):
        adg.probe_wait(0)
    with pytest.raises(adg.AdgError):
        adg.probe_wait(5_000_000_000)


@pytest.mark.parametrize("kw,msg", [
    (dict(dim=2, n_elem=(6, 6), P=(4, 4), flux="at", max_delay=2), "divide"),
    (dict(dim=2, n_elem=(8, 8), degree=0), "degree"),
    (dict(dim=2, n_elem=(8, 8), degree=8), "degree"),
    (dict(dim=3, n_elem=(2, 2, 2), degree=6), "3D"),
    (dict(dim=2, n_elem=(8, 8), flux="std", max_delay=0, P=(2, 2)), "max_delay"),
    (dict(dim=2, n_elem=(8, 8), flux="learned", max_delay=2, P=(2, 2), at_np=3), "at_np"),
    (dict(dim=2, n_elem=(8, 8), delay_mode="random", random_delay_max=16, flux="at",
          P=(2, 2), max_delay=2), "random_delay_max"),
    (dict(dim=2, n_elem=(8, 8), gamma=1.0), "gamma"),
    (dict(dim=2, n_elem=(8, 8), cfl=0.0, dt=0.0), "dt"),
])
def test_create_rejects_bad_configurations_without_gpu(kw, msg):
    # validation happens before any device work: status and message, no CUDA call
    with pytest.raises(adg.AdgError, match=msg) as e:
        adg.Solver(**kw)
    assert e.value.status in (1, 2)


def test_empty_and_null_inputs_without_gpu():
    import ctypes
    L = adg.lib()
    # an empty sample set is a no-op; missing buffers are refused
    assert L.adg_mlp_forward(None, None, 0, None, None) == 1  # NULL params: invalid
    p = (ctypes.c_uint16 * adg.lib().adg_mlp_num_params())()
    x = (ctypes.c_float * 4)()
    y = (ctypes.c_float * 1)()
    assert L.adg_mlp_forward(p, x, 0, y, None) == 0
    assert L.adg_mlp_grad(p, x, x, -1, y, y, None) == 1
    # batches need at least one instance; NULL handles are refused, destroy is NULL-safe
    h = ctypes.c_void_p()
    assert L.adg_batch_create(0, None, None, None, None, 2, None, ctypes.byref(h)) == 1
    assert L.adg_step(None, 1) == 1
    n = ctypes.c_int64()
    assert L.adg_checkpoint_bytes(None, ctypes.byref(n)) == 1
    assert L.adg_checkpoint_restore(None, None, 0) == 1
    L.adg_destroy(None)
    L.adg_batch_destroy(None)


def test_meshes_beyond_the_index_range_are_rejected_before_any_allocation():
    # 32-bit node indexing: (dim+2) * elements * (degree+1)^dim must stay below 2^31; the
    # check runs before the library touches the GPU (this test needs none)
    with pytest.raises(adg.AdgError) as e:
        adg.Solver(n_elem=(8192, 4096), degree=4)     # 4 * 33.5e6 * 25 = 3.4e9 DoF
    assert e.value.status == 2 and "2^31" in str(e.value)
    with pytest.raises(adg.AdgError) as e:
        adg.Solver(dim=3, n_elem=(512, 512, 256), degree=3)
    assert e.value.status == 2
    with pytest.raises(adg.AdgError):
        adg.Solver(n_elem=(8, 8), degree=8)           # degree 1..7 in 2D
    with pytest.raises(adg.AdgError):
        adg.Solver(n_elem=(8, 8), P=(2, 2), flux="at", max_delay=16)
    with pytest.raises(adg.AdgError):
        adg.Solver(n_elem=(8, 8), P=(2, 2), flux="at", delay_mode="random", random_delay_max=16)
