"""Run Alg. ConOptM on one of the synthetic systems from the command line.

  python -m paper_1308_2864_gb300.cli --config c2 --maxit 5 [--precision fp64|mixed]
                                      [--retraction qr|cayley] [--gtol 1e-6] [--verbose 0]
                                      [--N 40] [--p 512] [--fp64-emulation 0|1|2]

--N / --p shrink or change a configuration's grid and orbital count (same
cube, atoms and functional), e.g. to profile the p = 512 kernels of c3 on a
grid that fits a profiler's replay.

Prints one JSON line with the result (energy, ||D||_M, iterations, time).
Useful to profile a few iterations of the real workload.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None) -> int:
    import numpy as np
    import torch

    import ks_inputs as ki
    import paper_1308_2864_gb300 as ks

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--config", default="c2", choices=sorted(ki.CONFIGS))
    ap.add_argument("--maxit", type=int, default=300)
    ap.add_argument("--gtol", type=float, default=1e-6)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--retraction", default=None, choices=["qr", "cayley"])
    ap.add_argument("--verbose", type=int, default=0)
    ap.add_argument("--N", type=int, default=0, help="override the interior nodes per edge")
    ap.add_argument("--p", type=int, default=0, help="override the number of orbitals")
    ap.add_argument("--fp64-emulation", type=int, default=0, choices=[0, 1, 2],
                    help="FP64 Grams and updates on the tensor cores by digit splitting")
    a = ap.parse_args(argv)

    s = ki.CONFIGS[a.config]()
    if a.N > 0:
        s.N = a.N
    if a.p > 0:
        s.p = a.p
    P = ks.Problem.from_system(s)
    P.set_fp64_emulation(a.fp64_emulation)
    X = torch.from_numpy(np.ascontiguousarray(s.x0())).cuda()
    t0 = time.perf_counter()
    r = P.minimize(X, retraction=a.retraction or s.retraction, maxit=a.maxit, gtol=a.gtol,
                   precision=a.precision, verbose=a.verbose)
    torch.cuda.synchronize()
    r["wall_s"] = time.perf_counter() - t0
    r["config"] = a.config
    r["fp64_emulation"] = a.fp64_emulation
    print(json.dumps(r))
    return 0


if __name__ == "__main__":
    sys.exit(main())
