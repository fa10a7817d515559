"""Pins of the MLP oracle: analytic gradient against central finite differences, special
cases with closed forms, and BF16 rounding against its definition."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.3, mlp.N_PARAMS)
    x = rng.normal(0, 1, (37, 4))
    t = rng.normal(0, 1, 37)
    _, g = mlp.loss_and_grad(p, x, t)
    h = 1e-6
    idx = np.concatenate([rng.integers(0, mlp.N_PARAMS, 60), [0, 255, 256, 319, 320, 4415,
                                                                4416, 4479, 4480, 4543, 4544]])
    for i in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[i] = h
        fd = (mlp.loss_and_grad(p + e, x, t)[0] - mlp.loss_and_grad(p - e, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-7 * max(1.0, abs(fd)), i


def test_closed_forms():
    p = np.zeros(mlp.N_PARAMS)
    p[4544] = 0.75                          # only the output bias
    x = np.ones((5, 4))
    t = np.arange(5.0)
    y, _ = mlp.forward(p, x)
    assert np.all(y == 0.75)
    loss, g = mlp.loss_and_grad(p, x, t)
    assert np.isclose(loss, np.mean((0.75 - t) ** 2))
    assert np.isclose(g[4544], 2 * np.mean(0.75 - t))
    # with all hidden weights zero the hidden activations vanish, so only b2, w3 (through
    # tanh(b2) = 0) and b3 can move: their gradients are the only nonzero ones besides b2's
    assert np.all(g[:4480] == 0)


def test_bf16_rounding_definition():
    vals = np.array([1.0, 1.00390625, 1.001953125, -3.14159265, 1e-3, 65504.0], dtype=np.float32)
    r = mlp.bf16_round(vals)
    for v, q in zip(vals, r):
        # BF16 keeps 8 significant bits: q is the nearest such value (ties to even)
        e = np.floor(np.log2(abs(float(v))))
        step = 2.0 ** (e - 7)
        cands = np.floor(float(v) / step) * step + np.array([0.0, step])
        best = cands[np.argmin(np.abs(cands - float(v)))]
        assert q == best or abs(q - float(v)) == abs(best - float(v))
