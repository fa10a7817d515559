"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the method: it only draws numbers.  States are drawn
directly in conserved variables (rho, rho*u, E) inside ranges where the pressure stays
positive; vortex-instance parameters are drawn for the batched workload.
"""
from __future__ import annotations

import numpy as np


def random_state(shape, dim: int, seed: int = 0, rho=(0.8, 1.2), mom=(-0.3, 0.3),
                 energy=(2.3, 2.7)) -> np.ndarray:
    """Independent uniform draws per node: shape = (dim+2, n_elem, nodes_per_elem)."""
    rng = np.random.default_rng(seed)
    nv = dim + 2
    assert shape[0] == nv
    u = np.empty(shape)
    u[0] = rng.uniform(*rho, size=shape[1:])
    for d in range(dim):
        u[1 + d] = rng.uniform(*mom, size=shape[1:])
    u[nv - 1] = rng.uniform(*energy, size=shape[1:])
    return u


def vortex_instances(count: int = 64, seed: int = 7):
    """Parameter sets of the batched isentropic-vortex workload: strength beta ~ U[1, 5],
    centre ~ U([-2, 2]^2), mesh n^2 with n in {32, 64, 128, 256}, degree in {2..5},
    maximum delay L in {2, 3, 4}."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        out.append(dict(beta=float(rng.uniform(1.0, 5.0)),
                        x0=float(rng.uniform(-2.0, 2.0)), y0=float(rng.uniform(-2.0, 2.0)),
                        n=int(rng.choice([32, 64, 128, 256])), degree=int(rng.integers(2, 6)),
                        max_delay=int(rng.integers(2, 5))))
    return out


def vortex_params(count: int = 200, seed: int = 11):
    """(beta, centre) sets for the training runs of the learned predictor: beta ~ U[1, 5],
    centre ~ U([-2, 2]^2)."""
    rng = np.random.default_rng(seed)
    return [dict(beta=float(rng.uniform(1.0, 5.0)), x0=float(rng.uniform(-2.0, 2.0)),
                 y0=float(rng.uniform(-2.0, 2.0))) for _ in range(count)]
