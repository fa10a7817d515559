"""The fused per-stage kernel (one launch per RK stage: face fluxes, volume terms and the RK
update of a tile of elements, tiles staged by TMA tensor copies) against the split path
(face-flux launch + volume launch) and against the oracle.

FP64: the fused kernel evaluates every quantity with the same operations in the same order
as the split kernels (same traces, same face-flux code, same sweeps, lift and update), so
the two paths agree bit for bit.  FP32 pairs: the split path's 2D sweeps use packed
instructions with another summation order, so the paths agree to the pair arithmetic's
accuracy (1e-13 relative).  FP32: the split path interpolates the next stage's traces from
a fused-multiply-add form of the new solution, the fused path from its FP32 rounding (the
value the next stage loads), so the paths agree to FP32 accuracy.  Meshes cover whole and
ragged tiles, one tile spanning a whole periodic direction, and row lengths that rule out
TMA (the kernel then stages the tile with plain loads).
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


def run(path, precision, dim, n_elem, degree, steps, tgv=False, **kw):
    lo = (0.0,) * 3 if tgv else (-5.0,) * dim
    hi = (2 * np.pi,) * 3 if tgv else (5.0,) * dim
    s = adg.Solver(dim=dim, n_elem=n_elem, degree=degree, lo=lo, hi=hi, precision=precision,
                   kernel_path=path, **kw)
    if tgv:
        s.init_tgv(0.1)
    else:
        s.init_vortex(beta=3.0, x0=0.7, y0=-0.4)
    c0 = s.conservation()
    s.step(steps)
    u = s.get_state()
    c1 = s.conservation()
    s.close()
    return u, c0, c1


CASES_2D = [((16, 16), 4), ((8, 9), 2), ((13, 7), 3), ((5, 3), 4), ((12, 8), 1), ((8, 4), 5),
            ((6, 4), 6), ((4, 6), 7)]
MODES = [("sync", "caa", 1, "ck45"), ("at", "caa", 2, "ck45"), ("std", "caa", 3, "rk33"),
         ("at_trace", "caa", 2, "rk22"), ("at", "random", 0, "ck45")]


@pytest.mark.parametrize("n_elem,p", CASES_2D)
@pytest.mark.parametrize("flux,mode,L,rk", MODES)
def test_fused_fp64_equals_split_bitwise_2d(n_elem, p, flux, mode, L, rk):
    P = tuple(2 if n % 2 == 0 else 1 for n in n_elem)
    kw = dict(P=P, max_delay=L, flux=flux, rk=rk, delay_mode=mode, random_delay_max=2,
              seed=20260301, dt=0.004)
    a, _, _ = run("split", "fp64", 2, n_elem, p, 9, **kw)
    b, c0, c1 = run("fused", "fp64", 2, n_elem, p, 9, **kw)
    assert np.array_equal(a, b), rel(b, a)
    assert np.abs(c1 - c0).max() < 1e-12 * np.abs(c0).max()


@pytest.mark.parametrize("n_elem,p", [((4, 4, 4), 3), ((3, 2, 2), 2), ((5, 3, 4), 2),
                                      ((4, 4, 2), 1), ((2, 2, 2), 4), ((2, 2, 1), 5)])
@pytest.mark.parametrize("flux,mode,L,rk", [("at", "caa", 2, "ck45"), ("at_trace", "random", 0, "rk33")])
def test_fused_fp64_equals_split_bitwise_3d(n_elem, p, flux, mode, L, rk):
    P = tuple(2 if n % 2 == 0 else 1 for n in n_elem)
    kw = dict(P=P, max_delay=L, flux=flux, rk=rk, delay_mode=mode, random_delay_max=2,
              seed=7, dt=0.004)
    a, _, _ = run("split", "fp64", 3, n_elem, p, 7, tgv=True, **kw)
    b, c0, c1 = run("fused", "fp64", 3, n_elem, p, 7, tgv=True, **kw)
    assert np.array_equal(a, b), rel(b, a)
    assert np.abs(c1 - c0).max() < 1e-12 * np.abs(c0).max()


@pytest.mark.parametrize("precision,tol", [("df64", 1e-13), ("fp32", 1e-5)])
@pytest.mark.parametrize("dim,n_elem,p", [(2, (16, 16), 4), (2, (8, 9), 2), (2, (5, 3), 4),
                                          (3, (4, 4, 4), 3), (3, (3, 2, 2), 2)])
@pytest.mark.parametrize("flux,mode,L,rk", [("at", "caa", 2, "ck45"), ("std", "random", 0, "rk33")])
def test_fused_reduced_precision_matches_split(precision, tol, dim, n_elem, p, flux, mode, L, rk):
    P = tuple(2 if n % 2 == 0 else 1 for n in n_elem)
    kw = dict(P=P, max_delay=L, flux=flux, rk=rk, delay_mode=mode, random_delay_max=2,
              seed=3, dt=0.004)
    a, _, _ = run("split", precision, dim, n_elem, p, 8, tgv=dim == 3, **kw)
    b, c0, c1 = run("fused", precision, dim, n_elem, p, 8, tgv=dim == 3, **kw)
    assert rel(b, a) < tol
    # both sides of a face use the same flux bits, so the face terms cancel exactly; the
    # volume terms cancel only to the operator's rounding (FP32: the rounded derivative
    # weights no longer sum to zero; measured 4e-10 of the totals after 8 steps)
    assert np.abs(c1 - c0).max() < (1e-12 if precision == "df64" else 1e-8) * np.abs(c0).max()


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_fused_matches_oracle_bench_config(precision):
    # 2D p=4, N_p=4, L=3, 8x8 subdomains, CK4(5): two schedule cycles, states at 1e-12
    kw = dict(P=(8, 8), max_delay=3, flux="at", rk="ck45", dt=2e-3)
    s = adg.Solver(n_elem=(32, 32), degree=4, precision=precision, kernel_path="fused", **kw)
    o = O.Oracle(n_elem=(32, 32), degree=4, **kw)
    u0 = o.init_vortex()
    s.set_state(u0)
    o.set_state(u0)
    for n in range(16):
        s.step(1)
        o.step(1)
        assert rel(s.get_state(), o.get_state()) < 1e-12, n
    s.close()


def test_fused_checkpoint_continues_on_split_path():
    # a checkpoint of a fused-path handle carries every face trace, so a split-path handle
    # continues it exactly like the fused one
    kw = dict(n_elem=(16, 16), degree=3, P=(4, 4), max_delay=3, flux="at", rk="ck45", dt=3e-3)
    a = adg.Solver(kernel_path="fused", **kw)
    a.init_vortex()
    a.step(5)
    ck = a.checkpoint()
    a.step(6)
    ua = a.get_state()
    b = adg.Solver(kernel_path="split", **kw)
    b.restore(ck)
    b.step(6)
    assert np.array_equal(b.get_state(), ua)


def test_fused_handle_switching_to_the_split_path_mid_run():
    # trace logging and adg_rhs both need every face trace; a fused handle rebuilds them from
    # the solution before its next split-path step, so its run equals a split-path handle's
    import torch
    kw = dict(n_elem=(16, 16), degree=2, P=(4, 4), max_delay=2, flux="at", rk="ck45", dt=3e-3)
    runs = {}
    for path in ("split", "fused"):
        s = adg.Solver(kernel_path=path, **kw)
        s.init_vortex()
        s.step(4)
        u = s.get_state()
        s.rhs(u)                               # overwrites the current trace buffer
        s.step(3)
        rec = s.set_trace_log(None, 0)
        log = torch.zeros((12, rec), dtype=torch.float64, device="cuda")
        s.set_trace_log(log, 12)               # logging: the split path for these steps
        s.step(2)
        s.set_trace_log(None, 0)
        s.step(3)                              # back to the handle's own path
        runs[path] = (s.get_state(), log.cpu().numpy())
        s.close()
    assert np.array_equal(runs["split"][0], runs["fused"][0])
    assert np.array_equal(runs["split"][1], runs["fused"][1])
