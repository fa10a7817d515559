"""The paper's qualitative 2D results, rerun on the GPU operator (Section 5.3, Fig. 5 and the
stability remark that follows it).

Setting of Fig. 5: isentropic vortex on [-5, 5]^2, 64^2 quads (G = 4), 256 subdomains
(16 x 16 blocks of 4 x 4 elements), maximum delay L = 4, degree 2 with LSERK3, t_final = 4.

* `error_map` runs one scheme and returns the per-element maximum density error against
  the exact translating vortex, plus its summary numbers (the quantities Fig. 5 (d)-(f)
  shows as colour maps).
* `convergence_sweep` runs the isentropic vortex on a sequence of meshes with the
  synchronous, AT and standard delayed fluxes and returns the L2 errors and the observed
  orders (the degree-4 sweep of the 256^2 configuration: 32^2 .. 512^2, 8x8 subdomains,
  CAA L = 3, CK4(5)).
* `stability_limit` bisects the CFL number between a stable and an unstable value: the
  largest CFL number at which the scheme reaches t_final with a finite state.  The paper
  states that at L = 4 the standard-flux scheme becomes unstable at a CFL number at which
  the AT scheme is still stable; the CFL numbers themselves depend on the time-step rule,
  which the paper does not give (this library: dt = cfl h / ((2p+1) max(|u| + c))).
"""
import numpy as np

from . import adg

RK_OF_DEGREE = {1: "rk22", 2: "rk33"}


def _solver(n, degree, flux, cfl, t_final, P, max_delay, precision):
    return adg.Solver(n_elem=(n, n), degree=degree, P=(P, P), max_delay=max_delay, flux=flux,
                      rk=RK_OF_DEGREE[degree], cfl=cfl, t_end=t_final, precision=precision)


def run_vortex(flux, cfl, n=64, degree=2, t_final=4.0, P=16, max_delay=4, precision="fp64",
               keep_state=False):
    """Advance the vortex to t_final; returns dict(finite, steps, dt, l2[3], state?)."""
    s = _solver(n, degree, flux, cfl, t_final, P, max_delay, precision)
    try:
        s.init_vortex()
        dt = s.info()["dt"]
        steps = int(round(t_final / dt))
        s.step(steps)
        out = {"finite": bool(s.check_finite()), "steps": steps, "dt": dt}
        out["l2"] = s.l2_error_vortex(t_final) if out["finite"] else None
        if keep_state:
            out["state"] = s.get_state()
        return out
    finally:
        s.close()


def error_map(flux, cfl, n=64, degree=2, t_final=4.0, P=16, max_delay=4, precision="fp64"):
    """Per-element max |rho - rho_exact| at the nodes, shape (n, n) indexed [y][x], and
    summaries: max, mean over elements touching a subdomain face ("edge") and over the
    others ("inner"), and the L2 errors of density / momentum / energy."""
    r = run_vortex(flux, cfl, n, degree, t_final, P, max_delay, precision, keep_state=True)
    if not r["finite"]:
        return {"finite": False, "steps": r["steps"]}
    ex = _solver(n, degree, "sync", cfl, t_final, P, max_delay, precision)
    try:
        ex.init_vortex(t=t_final)
        exact = ex.get_state()
    finally:
        ex.close()
    emap = np.abs(r["state"][0] - exact[0]).max(axis=1).reshape(n, n)
    b = n // P
    i = np.arange(n)
    touches = (i % b == 0) | (i % b == b - 1)
    edge = touches[:, None] | touches[None, :]
    return {
        "finite": True, "steps": r["steps"], "dt": r["dt"], "l2": r["l2"], "map": emap,
        "max": float(emap.max()), "edge_mean": float(emap[edge].mean()),
        "inner_mean": float(emap[~edge].mean()) if (~edge).any() else float("nan"),
    }


def stability_limit(flux, lo, hi, iters=6, n=64, degree=2, t_final=4.0, P=16, max_delay=4,
                    precision="fp64"):
    """Bisection for the largest stable CFL number in [lo, hi]: `lo` must be stable and `hi`
    unstable (checked).  Returns (stable, unstable) after `iters` halvings."""
    ok = lambda c: run_vortex(flux, c, n, degree, t_final, P, max_delay, precision)["finite"]
    if not ok(lo) or ok(hi):
        raise ValueError(f"{flux}: [{lo}, {hi}] does not bracket the stability limit")
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if ok(mid):
            lo = mid
        else:
            hi = mid
    return lo, hi


def convergence_sweep(degree=4, meshes=(32, 64, 128, 256, 512), fluxes=("sync", "at", "std"),
                      P=8, max_delay=3, rk="ck45", cfl=0.1, t_final=1.0, precision="df64"):
    """L2 errors (density, momentum, energy) against the exact vortex at t_final for every
    flux and mesh, and the observed orders between successive meshes:
    {flux: {"n": [...], "steps": [...], "l2": [[3]...], "order": [[3]...]}}."""
    out = {}
    for flux in fluxes:
        rows = {"n": [], "steps": [], "l2": []}
        for n in meshes:
            s = adg.Solver(n_elem=(n, n), degree=degree, P=(P, P), max_delay=max_delay, flux=flux,
                           rk=rk, cfl=cfl, t_end=t_final, precision=precision)
            try:
                s.init_vortex()
                steps = int(round(t_final / s.info()["dt"]))
                s.step(steps)
                if not s.check_finite():
                    raise RuntimeError(f"{flux} {n}^2 diverged")
                rows["n"].append(n)
                rows["steps"].append(steps)
                rows["l2"].append([float(x) for x in s.l2_error_vortex(t_final)])
            finally:
                s.close()
        e = np.array(rows["l2"])
        rows["order"] = np.log2(e[:-1] / e[1:]).tolist()
        out[flux] = rows
    return out
