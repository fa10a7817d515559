"""Learned ghost-trace predictor: training data, training and evaluation.

Every arithmetic step runs in the library's CUDA kernels (trace logging, sample
construction, MLP forward/backward, Adam); torch only holds device buffers.

Recipe (the committed model ``trained/ghost_mlp.npz``); network inputs per scalar channel:
the two level differences in units of the level spread, the integer delay k / 8 and the RK
stage offset c_m; target: (truth - AT extrapolation) / (AT minus linear extrapolation), a
learned next-order step, kept where |target| <= 2:
  data   -- synchronous runs (AT-trace mode with L = 0, i.e. every step communicates) of the
            2D isentropic vortex on 256^2 quads, p = 4, 8x8 subdomains, CK4(5), CFL 0.1,
            with 200 seeded (beta, centre) sets; the subdomain-face traces of every stage
            are logged and samples drawn for delays k = 1..4 and every stage;
  model  -- 4 -> 64 -> 64 -> 1 MLP, tanh, BF16 weights / FP32 accumulation; Adam;
  use    -- ADG_FLUX_LEARNED with at_np = 2: correction of the AT trace extrapolation,
            AT itself as fallback and arbiter (include/adg.h).
"""
from __future__ import annotations

import argparse
import os

import numpy as np

from . import adg
from .inputs import vortex_params

HERE = os.path.dirname(os.path.abspath(__file__))
MODEL_PATH = os.path.join(HERE, "trained", "ghost_mlp.npz")
N_PARAMS = 4545


def init_params(seed=0):
    """Glorot-uniform weights, zero biases (FP32)."""
    rng = np.random.default_rng(seed)
    p = np.zeros(N_PARAMS, np.float32)
    a1 = np.sqrt(6.0 / (4 + 64))
    a2 = np.sqrt(6.0 / (64 + 64))
    a3 = np.sqrt(6.0 / (64 + 1))
    p[0:256] = rng.uniform(-a1, a1, 256)
    p[320:4416] = rng.uniform(-a2, a2, 4096)
    p[4480:4544] = rng.uniform(-a3, a3, 64)
    return p


class Trainer:
    """FP32 master weights, BF16 copy and Adam moments on the device."""

    def __init__(self, params_f32):
        import torch
        self.torch = torch
        self.p = torch.from_numpy(np.asarray(params_f32, np.float32).copy()).cuda()
        self.pbf = torch.empty(N_PARAMS, dtype=torch.int16, device="cuda")
        self.g = torch.zeros(N_PARAMS, dtype=torch.float32, device="cuda")
        self.m = torch.zeros_like(self.g)
        self.v = torch.zeros_like(self.g)
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.t = 0
        self.L = adg.lib()
        self._stream = torch.cuda.current_stream().cuda_stream
        adg._check(self.L.adg_mlp_to_bf16(self._ptr(self.p), self._ptr(self.pbf), self._stream))

    @staticmethod
    def _ptr(t):
        import ctypes
        return ctypes.c_void_p(t.data_ptr())

    def grad(self, x, target):
        """Accumulates the MSE gradient of (x, target) into self.g; returns the loss."""
        self.loss.zero_()
        adg._check(self.L.adg_mlp_grad(self._ptr(self.pbf), self._ptr(x), self._ptr(target),
                                       x.shape[0], self._ptr(self.g), self._ptr(self.loss),
                                       self._stream))
        return self.loss

    def adam(self, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.t += 1
        adg._check(self.L.adg_mlp_adam(self._ptr(self.p), self._ptr(self.pbf), self._ptr(self.g),
                                       self._ptr(self.m), self._ptr(self.v), lr, b1, b2, eps,
                                       self.t, self._stream))

    def forward(self, x):
        y = self.torch.empty(x.shape[0], dtype=self.torch.float32, device="cuda")
        adg._check(self.L.adg_mlp_forward(self._ptr(self.pbf), self._ptr(x), x.shape[0],
                                          self._ptr(y), self._stream))
        return y

    def params_bf16(self):
        return self.pbf.cpu().numpy().view(np.uint16).copy()

    def params_f32(self):
        return self.p.cpu().numpy().copy()


def run_samples(n_elem, degree, beta, x0, y0, steps, kmax, n_samples, rng, cfl=0.1, P=(8, 8)):
    """Synchronous run with trace logging; samples (x, target) for random channels, steps
    >= kmax + 2, stages and delays 1..kmax, built by the library's sample kernel."""
    import torch
    s = adg.Solver(n_elem=n_elem, degree=degree, P=P, max_delay=0, flux="at_trace", at_np=2,
                   rk="ck45", cfl=cfl)
    s.init_vortex(beta=beta, x0=x0, y0=y0)
    stages = 5
    rec_len = s.set_trace_log(None, 0)
    n_rec = steps * stages
    log = torch.empty(n_rec * rec_len, dtype=torch.float64, device="cuda")
    s.set_trace_log(log, n_rec)
    s.step(steps)
    s.set_trace_log(None, 0)
    picks = np.stack([rng.integers(0, rec_len, n_samples),
                      rng.integers(kmax + 2, steps, n_samples),
                      rng.integers(0, stages, n_samples),
                      rng.integers(1, kmax + 1, n_samples)], axis=1).astype(np.int32)
    pk = torch.from_numpy(picks).cuda()
    x = torch.empty((n_samples, 4), dtype=torch.float32, device="cuda")
    t = torch.empty(n_samples, dtype=torch.float32, device="cuda")
    ok = torch.empty(n_samples, dtype=torch.int32, device="cuda")
    s.learned_samples(log, n_rec, pk, x, t, ok)
    keep = ok.bool()
    s.close()
    return x[keep].contiguous(), t[keep].contiguous()


def dataset(n_runs=200, n_elem=(256, 256), degree=4, steps=12, kmax=4, per_run=20000, seed=11,
            target_bound=2.0):
    """Samples of all runs; targets beyond target_bound (outside the region where the solver
    would accept a correction, trust <= target_bound) are left out."""
    import torch
    rng = np.random.default_rng(seed + 1)
    xs, ts = [], []
    for prm in vortex_params(n_runs, seed):
        x, t = run_samples(n_elem, degree, prm["beta"], prm["x0"], prm["y0"], steps, kmax, per_run, rng)
        keep = t.abs() <= target_bound
        xs.append(x[keep])
        ts.append(t[keep])
    return torch.cat(xs).contiguous(), torch.cat(ts).contiguous()


def train(x, t, epochs=20, batch=65536, lr=1e-3, seed=0, log=None):
    import torch
    tr = Trainer(init_params(seed))
    n = x.shape[0]
    gen = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen).cuda()
        tot = 0.0
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            xb, tb = x[idx].contiguous(), t[idx].contiguous()
            loss = tr.grad(xb, tb)
            tr.adam(lr)
            tot += float(loss.item()) * len(idx)
        losses.append(tot / n)
        if log:
            log(f"epoch {ep}: mse {losses[-1]:.4e}")
    return tr, losses


def save(tr, path=MODEL_PATH, **meta):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, params_f32=tr.params_f32(), params_bf16=tr.params_bf16(),
             **{k: np.asarray(v) for k, v in meta.items()})


def load(path=MODEL_PATH):
    d = np.load(path)
    return d["params_bf16"], d


def main():
    ap = argparse.ArgumentParser(description="train the learned ghost-trace predictor")
    ap.add_argument("--runs", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--out", default=MODEL_PATH)
    a = ap.parse_args()
    x, t = dataset(n_runs=a.runs)
    q = np.percentile(t.cpu().numpy(), [1, 25, 50, 75, 99])
    print(f"{x.shape[0]} samples; target variance {float(t.var()):.4e}; "
          f"percentiles 1/25/50/75/99: {np.array2string(q, precision=4)}", flush=True)
    tr, losses = train(x, t, epochs=a.epochs, log=lambda m: print(m, flush=True))
    save(tr, a.out, losses=np.array(losses), n_samples=x.shape[0], runs=a.runs,
         target_var=float(t.var()))
    print("saved", a.out)


if __name__ == "__main__":
    main()
