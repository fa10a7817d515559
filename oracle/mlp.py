"""CPU oracle of the learned ghost-trace predictor's MLP -- TEST INFRASTRUCTURE.

Plain numpy in FP64, written from the chain rule: y = w3 . tanh(W2 tanh(W1 x + b1) + b2)
+ b3 and the gradient of the mean squared error over a sample set.  Parameters are used
exactly as given; pass BF16-rounded values (``bf16_round``) to mirror the GPU kernels,
which read BF16 weights and accumulate in FP32.  Pinned by central finite differences
(tests/test_oracle_mlp.py).

Layout of the 4545 parameters: W1[64][4] | b1[64] | W2[64][64] | b2[64] | w3[64] | b3.
"""
import numpy as np

N_PARAMS = 4545


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[0:256].reshape(64, 4), p[256:320], p[320:4416].reshape(64, 64), p[4416:4480],
            p[4480:4544], p[4544])


def forward(p, x):
    W1, b1, W2, b2, w3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.tanh(x @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ w3 + b3, (x, h1, h2)


def loss_and_grad(p, x, t):
    """MSE = mean((y - t)^2) and its gradient with respect to every parameter."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    y, (x, h1, h2) = forward(p, x)
    n = len(y)
    r = y - np.asarray(t, dtype=np.float64)
    loss = np.mean(r * r)
    dy = 2.0 * r / n                       # d loss / d y
    g_w3 = h2.T @ dy
    g_b3 = dy.sum()
    dz2 = np.outer(dy, w3) * (1.0 - h2 * h2)
    g_W2 = dz2.T @ h1
    g_b2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (1.0 - h1 * h1)
    g_W1 = dz1.T @ x
    g_b1 = dz1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, g


def bf16_round(a):
    """FP32 -> BF16 (round to nearest even) -> back to FP64 values."""
    f = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((f + 0x7FFF + ((f >> 16) & 1)) >> 16).astype(np.uint32) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits(a):
    f = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((f + 0x7FFF + ((f >> 16) & 1)) >> 16).astype(np.uint16)


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, ICLR 2015, Algorithm 1) in FP64."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
