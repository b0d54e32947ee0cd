"""Write tests/golden/config1_oracle.json from the oracle alone.

Workload: 4 x 4 x 4 hexes of the unit cube, +-10 % vertex perturbation (seed 0),
random renumbering and orientation, order n = 3, lambda = 0, manufactured
u* = sin(pi x) sin(pi y) sin(pi z), homogeneous Dirichlet on the whole boundary,
two-scale PCG to a relative residual of 1e-8.
Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from synth import lattice_hex_mesh, manufactured_s, manufactured_u  # noqa: E402
from oracle.problem import Problem  # noqa: E402


def main():
    mesh = lattice_hex_mesh(4, 0.1, 0)
    pr = Problem(mesh, 3, 0.0)
    b = pr.load(manufactured_s(pr.coords, 0.0))
    u, it, hist = pr.solve(b, rtol=1e-8)
    out = {
        "workload": "E=4 a=0.1 seed=0 n=3 lambda=0 Dirichlet, two-scale PCG rtol=1e-8",
        "n_dof": int(pr.G),
        "iterations": int(it),
        "residual_history": [float(h) for h in hist],
        "max_error_vs_manufactured": float(np.max(np.abs(u - manufactured_u(pr.coords)))),
        "solution_l2": float(np.linalg.norm(u)),
        "amg_sizes": [int(s) for s in pr.amg.sizes()],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config1_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, out["iterations"])


if __name__ == "__main__":
    main()
