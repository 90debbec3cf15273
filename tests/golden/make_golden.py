"""Writes the oracle's regression values for the 64x64 disk -> ellipse+blob workload.

The paper prints no numerical example (its figures are images only), so these
fixtures are not the paper's numbers: they are the FP64 oracle's own outputs,
written by this script, which calls nothing but ``oracle`` and the seeded input
generators.  They guard the oracle against silent drift between commits.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import phantoms  # noqa: E402


def compute():
    out = {}
    for tag, rnd in (("p0_zero", False), ("p0_random", True)):
        w = phantoms.disk_pair_64(random_p0=rnd)
        c, g = oracle.cost_and_grad(w.I0[0], w.J[0], w.p0[0], w.T, w.sigma,
                                    float(w.mu[0]), float(w.rho[0]), float(w.lam[0]))
        It, pt, _ = oracle.shoot(w.I0[0], w.p0[0], w.T, w.sigma, float(w.mu[0]), float(w.rho[0]))
        out[tag] = {
            "cost": [float(x) for x in c],
            "grad_l2": float(np.sqrt((g ** 2).sum())),
            "grad_sum": float(g.sum()),
            "grad_at": {"32,32": float(g[32, 32]), "10,50": float(g[10, 50]),
                        "0,0": float(g[0, 0])},
            "I_T_sum": float(It[-1].sum()),
            "p_T_l2": float(np.sqrt((pt[-1] ** 2).sum())),
        }
    # the variants at the random momentum: det momentum update, Eulerian and hybrid
    # schemes, and the deformation of the grid
    w = phantoms.disk_pair_64(random_p0=True)
    args = (w.I0[0], w.J[0], w.p0[0], w.T, w.sigma, float(w.mu[0]), float(w.rho[0]),
            float(w.lam[0]))
    for tag, kw in (("det", dict(p_update="det")), ("euler", dict(scheme="euler")),
                    ("hybrid", dict(scheme="hybrid"))):
        c, g = oracle.cost_and_grad(*args, **kw)
        out["p0_random_" + tag] = {"cost": [float(x) for x in c],
                                   "grad_l2": float(np.sqrt((g ** 2).sum())),
                                   "grad_at": {"32,32": float(g[32, 32]), "10,50": float(g[10, 50])}}
    wdef, jac = oracle.deformation(w.I0[0], w.p0[0], w.T, w.sigma, float(w.mu[0]), float(w.rho[0]))
    out["p0_random_deformation"] = {"phi_l2": float(np.sqrt((wdef ** 2).sum())),
                                    "jac_min": float(jac.min()), "jac_max": float(jac.max()),
                                    "jac_sum": float(jac.sum())}
    return out


if __name__ == "__main__":
    data = {
        "workload": "disk64: 64x64 disk r=18 -> ellipse 14x22 + blob r=8, T=10, sigma=3, "
                    "mu=0.1, rho=1, lambda=1e-3 (phantoms.disk_pair_64, seed 1001)",
        "source": "FP64 oracle (oracle/meta_oracle.c); the paper prints no numbers",
        "values": compute(),
    }
    with open(os.path.join(HERE, "disk64_oracle.json"), "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    print("wrote disk64_oracle.json")
