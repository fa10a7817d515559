"""Learned ghost-trace predictor: the GPU MLP kernels against the CPU oracle (forward,
MSE gradient, Adam), training, the trace log and sample builder, the AT fallback (a zero
network reproduces AT bit for bit), and what the trained network gains over plain AT on the
3D Taylor-Green case."""
import ctypes
import os

import numpy as np
import pytest

from oracle import mlp as OM
from paper_2603_28710_gb300 import adg, learned

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_28710_gb300 import build
    build.build()


def _data(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 1, (n, 4)).astype(np.float32)
    t = (np.sin(x[:, 0]) + 0.5 * x[:, 1] * x[:, 2] - 0.3 * x[:, 3]).astype(np.float32)
    return x, t


def test_gradient_and_forward_match_oracle():
    import torch
    p = learned.init_params(3) + np.random.default_rng(4).normal(0, 0.05, 4545).astype(np.float32)
    tr = learned.Trainer(p)
    x, t = _data(3000, 5)                       # 23 full chunks of 128 and a ragged tail
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    loss = float(tr.grad(xd, td).item())
    g = tr.g.cpu().numpy()
    pb = OM.bf16_round(p)                        # the kernels read BF16 weights
    lo, go = OM.loss_and_grad(pb, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - lo) < 1e-5 * lo
    scale = np.abs(go).max()
    assert np.abs(g - go).max() < 2e-5 * scale
    y = tr.forward(xd).cpu().numpy()
    yo, _ = OM.forward(pb, x.astype(np.float64))
    assert np.abs(y - yo).max() < 2e-5 * (1 + np.abs(yo).max())


def test_adam_matches_oracle_and_refreshes_bf16():
    import torch
    p = learned.init_params(7)
    tr = learned.Trainer(p)
    x, t = _data(512, 8)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    tr.grad(xd, td)
    g = tr.g.cpu().numpy().astype(np.float64)
    tr.adam(1e-2)
    p1, _, _ = OM.adam_step(p.astype(np.float64), g, 0.0, 0.0, 1, 1e-2)
    assert np.abs(tr.params_f32() - p1).max() < 1e-6
    assert np.array_equal(tr.params_bf16(), OM.bf16_bits(tr.params_f32()))
    assert np.all(tr.g.cpu().numpy() == 0)


def test_training_reduces_the_loss():
    import torch
    x, t = _data(20000, 9)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    _, losses = learned.train(xd, td, epochs=30, batch=2048, lr=3e-3)
    print("training mse by epoch:", np.array2string(np.array(losses)[[0, 9, 19, 29]], precision=4))
    assert losses[-1] < 0.1 * losses[0]


def test_samples_from_a_synchronous_run():
    import torch
    rng = np.random.default_rng(0)
    s = adg.Solver(n_elem=(16, 16), degree=2, P=(4, 4), max_delay=0, flux="at_trace", at_np=2,
                   rk="ck45", cfl=0.1)
    s.init_vortex(beta=3.0, x0=0.5, y0=-0.5)
    rec = s.set_trace_log(None, 0)
    assert rec == 2 * 4 * 128 * 3          # sides x vars x subdomain faces x face nodes
    log = torch.full((10 * 5 * rec,), float("nan"), dtype=torch.float64, device="cuda")
    s.set_trace_log(log, 10 * 5)
    s.step(10)
    L = log.cpu().numpy().reshape(50, rec)
    assert np.isfinite(L).all()
    picks = np.array([[c, st, m, k] for c, st, m, k in zip(rng.integers(0, rec, 200),
                      rng.integers(6, 10, 200), rng.integers(0, 5, 200), rng.integers(1, 5, 200))],
                     np.int32)
    x = torch.empty((200, 4), dtype=torch.float32, device="cuda")
    t = torch.empty(200, dtype=torch.float32, device="cuda")
    ok = torch.empty(200, dtype=torch.int32, device="cuda")
    s.learned_samples(log, 50, torch.from_numpy(picks).cuda(), x, t, ok)
    x, t, ok = x.cpu().numpy(), t.cpu().numpy(), ok.cpu().numpy()
    c_stage = adg.host_rk("ck45")[2]
    n_ok = 0
    for i, (c, st, m, k) in enumerate(picks):
        a = [L[(st - k - l) * 5, c] for l in range(3)]
        km = k + c_stage[m]
        w = adg.host_at_coeffs(2, km)
        E = np.dot(w, a)
        E2 = a[0] + km * (a[0] - a[1])
        est = E - E2                        # AT error estimate
        sp = abs(a[0] - a[1]) + abs(a[1] - a[2])
        if not abs(est) > 1e-9 * sum(abs(q) for q in a):
            assert ok[i] == 0               # AT exact to rounding: no sample
            continue
        n_ok += 1
        assert ok[i] == 1
        np.testing.assert_allclose(x[i], [(a[0] - a[1]) / sp, (a[1] - a[2]) / sp, k / 8,
                                          c_stage[m]], rtol=1e-6, atol=1e-7)
        # E carries rounding of order 1e-15 |a|, divided by an estimate of at least 1e-9 |a|
        np.testing.assert_allclose(t[i], (L[st * 5 + m, c] - E) / est, rtol=1e-5, atol=1e-5)
    assert n_ok > 100


def test_zero_network_reproduces_at_bitwise():
    zero = np.zeros(4545, np.uint16)
    kw = dict(n_elem=(16, 16), degree=3, P=(4, 4), max_delay=3, at_np=2, rk="ck45", cfl=0.1)
    a = adg.Solver(flux="at_trace", **kw)
    b = adg.Solver(flux="learned", **kw)
    b.set_learned_model(zero)
    for s in (a, b):
        s.init_vortex(beta=4.0)
        s.step(13)
    assert np.array_equal(a.get_state(), b.get_state())


def _tgv_error(flux, model=None, steps=24, precision="df64", trust=1.0):
    kw = dict(dim=3, n_elem=(64, 64, 64), degree=3, lo=(0, 0, 0), hi=(2 * np.pi,) * 3,
              P=(8, 8, 8), rk="ck45", cfl=0.1, precision=precision)
    ref = adg.Solver(flux="sync", **kw)
    ref.init_tgv(0.1)
    ref.step(steps)
    u_ref = ref.get_state()
    s = adg.Solver(flux=flux, max_delay=4, at_np=2, **kw)
    if model is not None:
        s.set_learned_model(model, trust)
    s.init_tgv(0.1)
    u0 = s.get_state()
    s.step(steps)
    return np.linalg.norm(s.get_state() - u_ref) / np.linalg.norm(u_ref - u0)


@pytest.mark.skipif(not os.path.exists(learned.MODEL_PATH), reason="no trained model committed")
def test_trained_network_against_plain_at_on_taylor_green():
    # trained on 2D vortex traces (256^2, p=4), evaluated on the 3D Taylor-Green vortex
    # (64^3, p=3, L=4): the gain is e_AT / e_learned (> 1 would be an improvement)
    # Measured: the network does not beat AT here (gain x0.35 at trust 1, x0.68 at 0.05):
    # AT's residual on this smooth flow is far below its own E3 - E2 error estimate, and the
    # network's prediction noise exceeds it.  The trust test bounds the harm: a tight trust
    # recovers the AT result.
    model, meta = learned.load()
    e_at = _tgv_error("at_trace")
    for trust in (1.0, 0.05, 0.001):
        e_ml = _tgv_error("learned", model, trust=trust)
        print(f"Taylor-Green 64^3 p=3, L=4, 24 steps, trust {trust}: relative delay error "
              f"AT {e_at:.4e}, learned {e_ml:.4e}, gain x{e_at / e_ml:.3f}")
        assert np.isfinite(e_ml)
    assert e_ml <= 1.05 * e_at
