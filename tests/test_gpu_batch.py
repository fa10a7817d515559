"""Batched solver (adg_batch_*): many uneven vortex instances in one CUDA-graph step.

The batched kernels run the single-instance element code of the split path (face-flux
launch + volume launch) or, for the FP32 operator by default, of the element path (one
volume launch whose elements evaluate their own faces' fluxes; same bits), so every
instance must equal a separate split-path solver handle bit for bit; one small instance is
also checked against the oracle.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_28710_gb300 import adg
from paper_2603_28710_gb300.inputs import vortex_instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_28710_gb300 import build
    build.build()


INSTANCES = [dict(n_elem=(16, 16), degree=2, P=(2, 2), max_delay=2, beta=5.0, x0=0.0, y0=0.0),
             dict(n_elem=(24, 24), degree=3, P=(4, 3), max_delay=3, beta=3.0, x0=1.0, y0=-1.0),
             dict(n_elem=(32, 16), degree=3, P=(2, 4), max_delay=4, beta=2.0, x0=-1.5, y0=0.5),
             dict(n_elem=(8, 8), degree=4, P=(2, 2), max_delay=2, beta=4.0, x0=0.3, y0=0.2),
             dict(n_elem=(20, 20), degree=5, P=(4, 4), max_delay=3, beta=1.5, x0=-0.5, y0=1.5),
             dict(n_elem=(12, 12), degree=2, P=(3, 3), max_delay=4, beta=2.5, x0=2.0, y0=-2.0)]


def singles_after(insts, steps, **kw):
    out = []
    for ins in insts:
        s = adg.Solver(n_elem=ins["n_elem"], degree=ins["degree"], P=ins["P"],
                       max_delay=ins["max_delay"], kernel_path="split", **kw)
        s.init_vortex(beta=ins["beta"], x0=ins["x0"], y0=ins["y0"])
        s.step(steps)
        out.append(s.get_state())
        s.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "df64", "fp32"])
@pytest.mark.parametrize("flux,mode", [("at", "caa"), ("std", "caa"), ("at_trace", "random")])
def test_batch_equals_separate_solvers_bitwise(precision, flux, mode):
    kw = dict(flux=flux, rk="ck45", cfl=0.1, precision=precision, delay_mode=mode,
              random_delay_max=2, seed=3)
    b = adg.Batch(INSTANCES, **kw)
    for i, ins in enumerate(INSTANCES):
        b.init_vortex(i, beta=ins["beta"], x0=ins["x0"], y0=ins["y0"])
    b.step(7)
    b.step(4)
    ref = singles_after(INSTANCES, 11, **kw)
    for i in range(len(INSTANCES)):
        assert b.info(i)["step"] == 11
        assert np.array_equal(b.get_state(i), ref[i]), f"instance {i}"
    b.close()


def test_batch_after_autotune_and_reset():
    kw = dict(flux="at", rk="rk33", cfl=0.1, precision="df64")
    b = adg.Batch(INSTANCES, **kw)
    tiles = b.autotune(trials=2)
    assert len(tiles) == len({ins["degree"] for ins in INSTANCES})
    assert all(t in (64, 128, 256) for t in tiles)
    with pytest.raises(adg.AdgError):
        b.step(1)                      # autotuning leaves no valid state
    for i, ins in enumerate(INSTANCES):
        b.init_vortex(i, beta=ins["beta"], x0=ins["x0"], y0=ins["y0"])
    b.step(9)
    ref = singles_after(INSTANCES, 9, **kw)
    for i in range(len(INSTANCES)):
        assert np.array_equal(b.get_state(i), ref[i]), f"instance {i}"


def test_batch_instance_matches_oracle():
    ins = INSTANCES[0]
    b = adg.Batch([ins], flux="at", rk="ck45", dt=0.01, precision="df64")
    b.init_vortex(0, beta=ins["beta"], x0=ins["x0"], y0=ins["y0"])
    b.step(10)
    o = O.Oracle(n_elem=ins["n_elem"], degree=ins["degree"], P=ins["P"],
                 max_delay=ins["max_delay"], flux="at", rk="ck45", dt=0.01)
    o.set_state(o.init_vortex(beta=ins["beta"], x0=ins["x0"], y0=ins["y0"]))
    o.step(10)
    u, uo = b.get_state(0), o.get_state()
    assert np.linalg.norm(u - uo) / np.linalg.norm(uo) < 1e-12


def test_sixty_four_uneven_vortex_instances():
    # batched workload: 64 vortices, beta in [1,5], centres in [-2,2]^2, meshes 32^2..256^2,
    # degrees 2..5, L in {2,3,4}; 8x8 subdomains; FP32 operator, FP64 accumulation
    specs = vortex_instances(64, seed=7)
    insts = [dict(n_elem=(s["n"], s["n"]), degree=s["degree"], P=(8, 8), max_delay=s["max_delay"])
             for s in specs]
    b = adg.Batch(insts, flux="at", rk="ck45", cfl=0.1, precision="fp32")
    b.autotune(trials=2)
    for i, s in enumerate(specs):
        b.init_vortex(i, beta=s["beta"], x0=s["x0"], y0=s["y0"])
    b.step(6)
    # the tuner may step the largest instances as separate handles while the others share
    # the graph's persistent launches: compare one of each size, and the ends
    big = next(i for i, s in enumerate(specs) if s["n"] == 256)
    small = next(i for i, s in enumerate(specs) if s["n"] == 32)
    for i in sorted({0, 17, 63, big, small}):
        s = specs[i]
        one = adg.Solver(n_elem=(s["n"], s["n"]), degree=s["degree"], P=(8, 8),
                         max_delay=s["max_delay"], flux="at", rk="ck45", cfl=0.1, precision="fp32",
                         kernel_path="split")
        one.init_vortex(beta=s["beta"], x0=s["x0"], y0=s["y0"])
        one.step(6)
        assert np.array_equal(b.get_state(i), one.get_state())
    for i in range(64):
        assert np.isfinite(b.get_state(i)).all()


@pytest.mark.parametrize("rk", ["rk22", "rk33", "ck45"])
@pytest.mark.parametrize("path", ["auto", "split"])
def test_fp32_batch_paths_equal_separate_solvers(rk, path):
    # FP32: the element path by default (traces cycling through two buffers for an even
    # stage count, three for an odd one, back to the instance's own at the end of a step),
    # the split path on request; both give the split path's bits
    kw = dict(flux="at", rk=rk, cfl=0.1, precision="fp32")
    b = adg.Batch(INSTANCES, kernel_path=path, **kw)
    for i, ins in enumerate(INSTANCES):
        b.init_vortex(i, beta=ins["beta"], x0=ins["x0"], y0=ins["y0"])
    b.step(5)
    b.step(6)
    ref = singles_after(INSTANCES, 11, **kw)
    for i in range(len(INSTANCES)):
        assert np.array_equal(b.get_state(i), ref[i]), f"instance {i}"
    b.close()


def test_fp32_element_batch_after_autotune():
    # the tuner's separate-handle trials step instances on the element path (which swaps the
    # handle's trace buffers); states set afterwards give the batch its buffers back
    specs = vortex_instances(12, seed=5)
    insts = [dict(n_elem=(s["n"], s["n"]), degree=s["degree"], P=(8, 8), max_delay=s["max_delay"])
             for s in specs]
    kw = dict(flux="at", rk="ck45", cfl=0.1, precision="fp32")
    b = adg.Batch(insts, **kw)
    b.autotune(trials=2)
    for i, s in enumerate(specs):
        b.init_vortex(i, beta=s["beta"], x0=s["x0"], y0=s["y0"])
    b.step(3)
    b.step(4)
    for i, s in enumerate(specs):
        one = adg.Solver(n_elem=(s["n"], s["n"]), degree=s["degree"], P=(8, 8),
                         max_delay=s["max_delay"], kernel_path="split", **kw)
        one.init_vortex(beta=s["beta"], x0=s["x0"], y0=s["y0"])
        one.step(7)
        assert np.array_equal(b.get_state(i), one.get_state()), f"instance {i}"
        one.close()
    b.close()


@pytest.mark.parametrize("precision,rk", [("fp32", "ck45"), ("fp32", "rk22"), ("fp64", "ck45"),
                                          ("df64", "rk33")])
def test_3d_batch_equals_separate_solvers(precision, rk):
    # 3D Taylor-Green instances of degrees 1-3 (FP32: the batched element path; FP64 and
    # pairs: the split pair), against separate split-path handles, bit for bit
    box = dict(lo=(0.0, 0.0, 0.0), hi=(2 * np.pi,) * 3)
    insts = [dict(n_elem=(4, 4, 4), degree=3, P=(2, 2, 2), max_delay=4, **box),
             dict(n_elem=(6, 4, 2), degree=2, P=(2, 2, 1), max_delay=2, **box),
             dict(n_elem=(4, 4, 4), degree=2, P=(2, 2, 2), max_delay=3, **box),
             dict(n_elem=(2, 2, 2), degree=1, P=(1, 1, 1), max_delay=1, **box)]
    kw = dict(flux="at", rk=rk, cfl=0.1, precision=precision)
    b = adg.Batch(insts, dim=3, **kw)
    ones = []
    for i, ins in enumerate(insts):
        one = adg.Solver(dim=3, n_elem=ins["n_elem"], degree=ins["degree"], P=ins["P"],
                         max_delay=ins["max_delay"], lo=box["lo"], hi=box["hi"],
                         kernel_path="split", **kw)
        one.init_tgv(0.1)
        b.set_state(i, one.get_state())
        ones.append(one)
    b.step(6)
    for i, one in enumerate(ones):
        one.step(6)
        assert np.array_equal(b.get_state(i), one.get_state()), f"instance {i}"
        one.close()
    b.close()
