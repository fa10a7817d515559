"""Run one operator case for a profiler: build a solver, set the initial condition, advance.

    python -m paper_2603_28710_gb300.profile_case --dim 2 --n 512 --degree 4 \
        --precision fp32 --steps 2

2D: isentropic vortex on [-5, 5]^2; 3D: Taylor-Green vortex (Mach 0.1) on [0, 2 pi]^3.
P x P (x P) subdomains, maximum delay L, AT flux, CK4(5), CFL 0.1.  Prints one line.
"""
import argparse
import math


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dim", type=int, default=2, choices=[2, 3])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--degree", type=int, default=4)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "df64"])
    ap.add_argument("--flux", default="at")
    ap.add_argument("--P", type=int, default=8)
    ap.add_argument("--L", type=int, default=3)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--path", default="auto", choices=["auto", "split", "fused", "element"])
    a = ap.parse_args(argv)
    import torch
    from . import adg
    d = a.dim
    box = ((-5.0,) * d, (5.0,) * d) if d == 2 else ((0.0,) * d, (2 * math.pi,) * d)
    s = adg.Solver(dim=d, n_elem=(a.n,) * d, lo=box[0], hi=box[1], degree=a.degree, P=(a.P,) * d,
                   max_delay=a.L, flux=a.flux, rk="ck45", cfl=0.1, precision=a.precision,
                   kernel_path=a.path)
    if d == 2:
        s.init_vortex()
    else:
        s.init_tgv(0.1)
    s.step(a.steps)
    torch.cuda.synchronize()
    print(f"profile_case dim={d} n={a.n} p={a.degree} {a.precision} path={a.path} steps={a.steps} "
          f"dof={s.n_dof} finite={s.check_finite()}")
    s.close()


if __name__ == "__main__":
    main()
