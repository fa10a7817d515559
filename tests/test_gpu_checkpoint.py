"""Checkpoint / resume through the C ABI (adg_checkpoint_*): a run split by a checkpoint,
restored into a fresh handle, equals the straight run bit for bit, in every flux mode,
delay mode and operator arithmetic; incompatible or damaged checkpoints are refused."""
import numpy as np
import pytest

from paper_2603_28710_gb300 import adg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_28710_gb300 import build
    build.build()


def make(**kw):
    base = dict(n_elem=(16, 16), degree=2, P=(4, 4), max_delay=3, flux="at", rk="ck45",
                cfl=0.2, precision="fp64")
    base.update(kw)
    return adg.Solver(**base)


CASES = [
    dict(flux="at"),
    dict(flux="std"),
    dict(flux="at_trace"),
    dict(flux="sync"),
    dict(flux="at", rk="rk33"),
    dict(flux="at", delay_mode="random", random_delay_max=2, seed=1234),
    dict(flux="at", precision="df64"),
    dict(flux="at", precision="fp32"),
    dict(flux="std", precision="fp32", rk="rk22"),
    dict(flux="at", dim=3, n_elem=(8, 8, 8), lo=(0, 0, 0), hi=(1, 1, 1), P=(2, 2, 2), degree=2),
]


@pytest.mark.parametrize("kw", CASES, ids=lambda k: "-".join(f"{a}={b}" for a, b in k.items()))
@pytest.mark.parametrize("split", [1, 5, 9])
def test_split_run_equals_straight_run(kw, split):
    total = 12
    a = make(**kw)
    if a.dim == 3:
        rng = np.random.default_rng(5)
        u0 = np.empty(a.shape)
        u0[0] = 1.0 + 0.1 * rng.random(u0[0].shape)
        u0[1:-1] = 0.1 * rng.standard_normal(u0[1:-1].shape)
        u0[-1] = 2.5 + 0.1 * rng.random(u0[-1].shape)
        a.set_state(u0)
    else:
        a.init_vortex()
    a.step(total)
    straight = a.get_state()
    t_straight = a.info()
    a.close()

    b = make(**kw)
    if b.dim == 3:
        b.set_state(u0)
    else:
        b.init_vortex()
    b.step(split)
    ck = b.checkpoint()
    b.close()
    c = make(**kw)
    c.restore(ck)
    assert c.info()["step"] == split
    c.step(total - split)
    resumed = c.get_state()
    info = c.info()
    c.close()
    assert np.array_equal(resumed, straight)
    assert info["step"] == t_straight["step"] and info["t"] == t_straight["t"]


def test_checkpoint_refused_when_incompatible_or_damaged():
    a = make(flux="at")
    a.init_vortex()
    a.step(3)
    ck = a.checkpoint()
    a.close()
    for kw, field in [(dict(flux="std"), "flux"), (dict(max_delay=2), "max_delay"),
                      (dict(precision="df64"), "precision"), (dict(degree=3), "degree"),
                      (dict(P=(2, 2)), "P"), (dict(n_elem=(32, 32)), "mesh")]:
        b = make(**kw)
        with pytest.raises(adg.AdgError, match=field):
            b.restore(ck)
        b.close()
    b = make(flux="at")
    with pytest.raises(adg.AdgError, match="truncated"):
        b.restore(ck[:-8])
    bad = ck.copy()
    bad[0] ^= 0xFF
    with pytest.raises(adg.AdgError, match="not an ADG checkpoint"):
        b.restore(bad)
    with pytest.raises(adg.AdgError):  # nothing to save before a state exists
        b.checkpoint()
    b.close()


def test_resume_without_ring_restarts_the_warm_up():
    # restarting from the state alone (adg_set_state) is a new run: its schedule starts at
    # step 0 with the communication steps of Algorithm 3's warm-up
    a = make(flux="at")
    a.init_vortex()
    a.step(4)
    u = a.get_state()
    a.set_state(u)
    comm, k, _ = a.schedule(0, 3)
    assert a.info()["step"] == 0 and list(comm) == [1, 1, 1]
    a.close()
