"""Write the oracle's preconditioned GMRES(50) iteration counts for the 64^3 sweep.

Test infrastructure only: calls nothing but the oracle and the seeded input
generators.  Output: tests/golden/config2_oracle_iters.txt, one line per
(box, refractive index, right-hand side) with the iteration count of the
3-level-preconditioned (restricted to the scatterer) right-preconditioned
GMRES(50) at relative residual 1e-6 and the final true residual.

    python -m oracle.iteration_counts
"""
from __future__ import annotations

import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from dda_inputs import config2_cases  # noqa: E402
from oracle.problem import from_case  # noqa: E402
import numpy as np  # noqa: E402


def main():
    out = os.path.join(ROOT, "tests", "golden", "config2_oracle_iters.txt")
    lines = ["# Oracle (CPU FP64) right-preconditioned GMRES(50), 3-level circulant",
             "# preconditioner restricted to the scatterer, tol 1e-6, x0 = 0.",
             "# 64^3 hexagonal prisms, x = 20, seeded direction (seed 0), polarisations e1, e2.",
             "# Written by oracle/iteration_counts.py.",
             "# l m n eps_re eps_im rhs iters rel_resid"]
    for case in config2_cases(64, 20.0, seed=0):
        eps = complex(case.eps[0])
        if abs(eps - 1.78 ** 2) < 1e-9:
            continue
        for r in range(case.nrhs):
            prob = from_case(case, r)
            t0 = time.time()
            x, info = prob.solve_gmres("3", tol=1e-6, restart=50, maxiter=2000)
            res = np.linalg.norm(prob.rhs() - prob.matvec(x)) / np.linalg.norm(prob.rhs())
            l, m, n = case.dims
            lines.append(f"{l} {m} {n} {eps.real:.6f} {eps.imag:.6f} {r} {info['iters']} {res:.3e}")
            print(lines[-1], f"({time.time() - t0:.0f} s)", flush=True)
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
