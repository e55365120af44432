"""Orbital-free (Thomas-Fermi-von Weizsaecker) aluminium-like clusters: time
to ||grad||_M <= gtol of Alg. ConOptM on the unit sphere of the M metric
(Eq. OFDFT-y, p = 1), the model and criterion of the paper's orbital-free
runs (Sec. 5, which stops at ||grad|| <= 1e-5).

  python -m paper_1308_2864_gb300.of_bench --cells 4 --retraction qr --precision fp64

Workload: the fcc cluster recipe of ks_inputs.config_of_al (s x s x s cubic
cells of edge 7.559 bohr, every lattice point of the block, Z = 3 erf
pseudo-atoms, 6 bohr of vacuum, spacing 0.4 bohr).  One JSON line per run.
"""
from __future__ import annotations

import argparse
import json
import time

HARTREE_EV = 27.211386245988


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--cells", type=int, default=4)
    ap.add_argument("--mu", type=float, default=1.0)
    ap.add_argument("--spacing", type=float, default=0.4)
    ap.add_argument("--retraction", default="qr", choices=["qr", "cayley"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--gtol", type=float, default=1e-5)
    ap.add_argument("--maxit", type=int, default=5000)
    ap.add_argument("--repeat", type=int, default=1, help="solves from the same start (timed each)")
    ap.add_argument("--save", default="", help="write the final amplitude (n x 1, .npy)")
    ap.add_argument("--N", type=int, default=0, help="grid nodes per edge (spacing follows)")
    ap.add_argument("--levels", type=int, default=1,
                    help="uniform refinement: solve on N_0 = (N+1)/2^(levels-1) - 1 first")
    ap.add_argument("--coarse-gtol", type=float, default=1e-3)
    a = ap.parse_args(argv)

    import numpy as np
    import torch

    import ks_inputs as ki
    import paper_1308_2864_gb300 as ks

    s = ki.config_of_al(cells=a.cells, spacing=a.spacing, mu=a.mu, N=a.N or None)
    torch.cuda.init()
    if a.levels > 1:
        return refine(a, s)
    t0 = time.perf_counter()
    P = ks.Problem.from_system(s)
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    x0 = torch.from_numpy(np.ascontiguousarray(s.x0())).cuda()
    times, res = [], None
    for _ in range(max(1, a.repeat)):
        c = x0.clone()
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = P.minimize(c, retraction=a.retraction, gtol=a.gtol, maxit=a.maxit,
                         precision=a.precision)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
    natoms = len(s.atoms)
    out = {"workload": s.name, "cells": a.cells, "atoms": natoms, "N": s.N, "n": s.n,
           "mu": a.mu, "retraction": a.retraction, "precision": a.precision, "gtol": a.gtol,
           "setup_s": round(setup, 3), "solve_s": [round(x, 4) for x in times],
           "status": res["status"], "iters": res["iters"], "backtracks": res["backtracks"],
           "cg_iters_total": res["cg_iters_total"], "gradnorm": res["gradnorm"],
           "E_ha": res["E"], "E_per_atom_ev": res["E"] * HARTREE_EV / natoms,
           "E_parts_ha": dict(zip(["kinetic", "external", "hartree", "xc", "ion"],
                                  [float(v) for v in res["E_parts"]])),
           "mixed_iters": res.get("mixed_iters", 0),
           "ms_per_iter": round(1e3 * min(times) / max(1, res["iters"]), 4)}
    if a.save:
        np.save(a.save, c.cpu().numpy())
    print(json.dumps(out), flush=True)
    P.close()
    return 0


def refine(a, s) -> int:
    """Alg. AdpConOptM with uniform refinement, timed end to end (problem
    set-up of every level included) against nothing else: the single-grid
    solve is the same command without --levels."""
    import numpy as np
    import torch

    import paper_1308_2864_gb300 as ks

    grids = ks.refine_grids(s.N, a.levels)
    times, res = [], None
    for _ in range(max(1, a.repeat)):
        torch.cuda.synchronize()
        t = time.perf_counter()
        res, _ = ks.minimize_refine(s, a.levels, coarse_gtol=a.coarse_gtol, want_x=False,
                                    retraction=a.retraction, gtol=a.gtol, maxit=a.maxit,
                                    precision=a.precision)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
    natoms = len(s.atoms)
    fin = res[-1]
    out = {"workload": s.name, "cells": a.cells, "atoms": natoms, "grids": grids,
           "levels": a.levels, "coarse_gtol": a.coarse_gtol, "mu": a.mu,
           "retraction": a.retraction, "precision": a.precision, "gtol": a.gtol,
           "wall_s": [round(x, 4) for x in times],
           "level_s": [round(r["seconds"], 4) for r in res],
           "level_iters": [r["iters"] for r in res],
           "level_backtracks": [r["backtracks"] for r in res],
           "status": fin["status"], "gradnorm": fin["gradnorm"], "E_ha": fin["E"],
           "E_per_atom_ev": fin["E"] * HARTREE_EV / natoms}
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
