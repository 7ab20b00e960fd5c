"""Writes tests/golden/full_size_valve32.json: the oracle's FGMRES iteration
count on the 3D valve workload (32^3 fine hexahedra, 4 levels, 1.69 M
unknowns, field-split blocks of one pressure vertex, omega = 0.7: the
configuration bench.py's valve3d leg times), which the oracle cannot
recompute inside a GPU test in reasonable time.

Stored value (from oracle/ on the seeded inputs of
paper_1909_13201_gb300/inputs.py; nothing from the CUDA path): the FGMRES(30)
iteration count to the float64 true relative residual 1e-8 with the GMG
preconditioner in the float16 row-scaled storage emulation (float64 inverses
rounded to float16 with a float32 row scale, float32 cycle, float64 Krylov),
additive field-split smoother.

Run from the repository root:  python tests/golden/make_full_size_reference_3d.py
(a few hours on one core, ~35 GB of memory).
"""
import json
import os
import sys
import time

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "..")))

from oracle import fgmres, gmg, mesh  # noqa: E402
from paper_1909_13201_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "full_size_valve32.json")


def main():
    p = I.make_config(2)
    lev = mesh.build_levels(p)[-1]
    b = I.gather_natural(I.natural_vector(p, 1), lev.dof_field, lev.dof_comp, lev.dof_node)
    out = {"workload": p.name, "n": int(b.size), "rhs": "gather_natural(natural_vector(make_config(2), 1))",
           "patch": int(p.patch), "omega": float(p.omega), "rtol": 1e-8}
    t = time.time()
    H = gmg.Hierarchy(p, mixed="half")
    print("hierarchy", f"{time.time() - t:.0f} s", flush=True)
    x, st = fgmres.solve(H, b, rtol=1e-8)
    assert st["converged"], st
    out["iterations_half_additive"] = int(st["iterations"])
    out["iterations_half_additive_rel_residual"] = float(st["rel_residual"])
    print("iterations_half_additive", st["iterations"], st["rel_residual"], f"{time.time() - t:.0f} s", flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
