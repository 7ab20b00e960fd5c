"""Run a few solves of one workload, for profiler captures (ncu).

    python -m paper_1909_13201_gb300.profile_case --config 4 --precision half --solves 2 --mult-levels 1
    python -m paper_1909_13201_gb300.profile_case --config 1 --mult-levels 1 --nonlinear 1

Builds nothing and times nothing: it sets up the hierarchy and smoothers of
the chosen workload and runs `--solves` FGMRES solves to 1e-8 from zero, so a
profiler sees exactly the solve kernels after a short set-up.  With
`--nonlinear STEPS` it runs that many implicit time steps of the nonlinear
problem (Sec. 2.2, body force 20) from rest instead: per Newton step the
Jacobians on every level, the blocks' refactorisation and one solve.
"""
from __future__ import annotations

import argparse

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", type=int, default=4)
    ap.add_argument("--precision", choices=["fp64", "mixed", "half"], default="half")
    ap.add_argument("--solves", type=int, default=2)
    ap.add_argument("--adjoint", action="store_true")
    ap.add_argument("--mult-levels", type=int, default=0,
                    help="finest levels smoothed by the multiplicative sweep (0: additive)")
    ap.add_argument("--nonlinear", type=int, default=0, help="implicit nonlinear time steps instead of solves")
    a = ap.parse_args()
    import torch

    from . import inputs as I
    from .binding import FSI_FP64, FSI_MIXED, FSI_MIXED_HALF, FSISolver
    prec = {"fp64": FSI_FP64, "mixed": FSI_MIXED, "half": FSI_MIXED_HALF}[a.precision]
    p = I.make_config(a.config)
    s = FSISolver(p, nonlinear=a.nonlinear > 0)
    s.setup_smoothers(precision=prec, mult_levels=a.mult_levels)
    lv = p.n_levels - 1
    if a.nonlinear > 0:
        s.nl_setup(force=20.0)
        n = s.sizes(lv)["n"]
        Un = torch.zeros(n, dtype=torch.float64, device="cuda")
        U = torch.empty_like(Un)
        for k in range(a.nonlinear):
            U.copy_(Un)
            g = s.nl_step(Un, U, (k + 1) * p.dt)
            Un.copy_(U)
        torch.cuda.synchronize()
        print(f"{p.name}: {a.nonlinear} nonlinear step(s), Newton {g['newton_steps']}, iterations {g['iterations']}")
        return
    f, c, nd = s.dof_map(lv)
    b = torch.from_numpy(I.gather_natural(I.natural_vector(p, 1), f.astype(np.int64), c.astype(np.int64),
                                          nd.astype(np.int64))).cuda()
    for _ in range(a.solves):
        x, st = s.solve(b, rtol=1e-8)
        if a.adjoint:
            s.adjoint(b, x, rtol=1e-8)
    torch.cuda.synchronize()
    print(f"{p.name}: {a.solves} solve(s), {st['iterations']} iterations, {st['solve_ms']:.1f} ms last")


if __name__ == "__main__":
    main()
