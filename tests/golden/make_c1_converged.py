"""Write c1_converged.json: the oracle's converged solution of the 24^3,
two-atom, p = 4 system (Slater exchange, Cayley step, Eq. WY3) to
||D||_M <= 1e-6 (Alg. ConOptM's stopping test in the M metric).

Only the oracle and the seeded input recipe are used.  Stored: the energy
and its parts, the spectrum of the Lagrange multipliers
Lambda = sym(X^T E_X) (at a KKT point H X = M X Lambda/(2f), so these are
2f times the occupied orbital energies), and the nodal density at a fixed
sample of nodes (the 128 densest nodes and 384 seeded random ones).  The
energy is also stored for the run that takes the rounding slack in the
Armijo test, to show that reading does not move the minimiser.

  python tests/golden/make_c1_converged.py        (about two minutes)
"""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import ks_inputs as ki  # noqa: E402
from oracle import energy as oe  # noqa: E402
from oracle import stiefel as ost  # noqa: E402

GTOL = 1e-6


def main():
    s = ki.config_c1()
    model = oe.Model.from_system(s)
    out = {"system": "c1: 24^3 interior nodes, L = 10 bohr, 2 atoms Z = 4, rc = 0.5, p = 4, "
                     "Slater exchange, Cayley retraction, ||D||_M <= 1e-6",
           "gtol": GTOL}
    r = ost.minimize(model, s.x0(), ost.Options(retraction="cayley", gtol=GTOL, maxit=20000))
    assert r.converged
    Lam = r.X.T @ r.point.ev.EX
    rho = oe.density(r.X, model.occ)
    rng = ki.SplitMix64(ki.stream_key(2024, 0, 7))
    dense = np.argsort(rho)[::-1][:128]
    rand = sorted({int(rng.uniform() * rho.size) for _ in range(384)} - set(dense.tolist()))
    nodes = sorted(set(dense.tolist()) | set(rand))
    out.update({
        "E": r.E, "parts": r.parts, "dnorm": r.dnorm, "iters": r.iters,
        "lambda_eigs": np.linalg.eigvalsh(0.5 * (Lam + Lam.T)).tolist(),
        "rho_max": float(rho.max()), "rho_sum_h3": float(rho.sum() * model.h ** 3),
        "rho_nodes": nodes, "rho_values": [float(rho[k]) for k in nodes],
    })
    rs = ost.minimize(model, s.x0(), ost.Options(retraction="cayley", gtol=GTOL, maxit=20000,
                                                 armijo_slack=True))
    assert rs.converged
    out["E_with_armijo_slack"] = rs.E
    out["iters_with_armijo_slack"] = rs.iters
    with open(os.path.join(HERE, "c1_converged.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(f"E = {r.E!r} ({r.iters} iterations), with slack {rs.E!r} ({rs.iters})")


if __name__ == "__main__":
    main()
