"""Run Alg. ConOptM on one of the synthetic systems from the command line.

  python -m paper_1308_2864_gb300.cli --config c2 --maxit 5 [--precision fp64|mixed]
                                      [--retraction qr|cayley] [--gtol 1e-6] [--verbose 0]
                                      [--N 40] [--p 512] [--fp64-emulation 0|1|2]
                                      [--profile 40] [--tensor-cores 0|1|2|3]

--N / --p shrink or change a configuration's grid and orbital count (same
cube, atoms and functional), e.g. to profile the p = 512 kernels of c3 on a
grid that fits a profiler's replay.

Prints one JSON line with the result (energy, ||D||_M, iterations, time).
Useful to profile a few iterations of the real workload.  --profile W runs W
iterations first, then resumes for --maxit more with the library's kernel
classes timed by CUDA events on the problem's stream, and adds to the line
the milliseconds per iteration and, per class, the launches and microseconds
per iteration.
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
    ap.add_argument("--tensor-cores", type=int, default=1, choices=[0, 1, 2, 3],
                    help="tensor-core use of the FP32 phase (ks_set_tensor_cores)")
    ap.add_argument("--profile", type=int, default=0, metavar="W",
                    help="time the kernel classes over --maxit iterations after W untimed ones")
    a = ap.parse_args(argv)

    s = ki.CONFIGS[a.config]()
    if a.N > 0:
        s.N = a.N
    if a.p > 0:
        s.p = a.p
    P = ks.Problem.from_system(s)
    P.set_fp64_emulation(a.fp64_emulation)
    P.set_tensor_cores(a.tensor_cores)
    X = torch.from_numpy(np.ascontiguousarray(s.x0())).cuda()
    kw = dict(retraction=a.retraction or s.retraction, gtol=a.gtol, precision=a.precision,
              verbose=a.verbose)
    prof = None
    if a.profile > 0:
        # warm-up, then the timed iterations resume the saved loop state
        # (the stall test off, so that both runs do the iterations asked for)
        P.minimize(X, maxit=a.profile, stall_iters=0, **kw)
        torch.cuda.synchronize()
        ks.profile_start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(P.stream)
        t0 = time.perf_counter()
        r = P.minimize(X, maxit=a.profile + a.maxit, stall_iters=0, resume=1, **kw)
        e1.record(P.stream)
        e1.synchronize()
        prof = ks.profile_stop()
        it = max(1, r["iters"])
        r["profile"] = {"iters": r["iters"], "ms_per_iter": e0.elapsed_time(e1) / it,
                        "classes": {k: {"launches_per_iter": n / it, "us_per_iter": 1e3 * ms / it}
                                    for k, (ms, n, _, _) in prof.items() if n}}
    else:
        t0 = time.perf_counter()
        r = P.minimize(X, maxit=a.maxit, **kw)
    torch.cuda.synchronize()
    r["wall_s"] = time.perf_counter() - t0
    r["config"] = a.config
    r["fp64_emulation"] = a.fp64_emulation
    r["tensor_cores"] = a.tensor_cores
    print(json.dumps(r))
    return 0


if __name__ == "__main__":
    sys.exit(main())
