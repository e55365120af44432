"""Batched and served minimisation jobs through the continuous-batching server.

  python -m paper_1308_2864_gb300.serve_bench --workload c4 --jobs 256 --slots 32
  python -m paper_1308_2864_gb300.serve_bench --workload c5 --jobs 64 --rate-frac 0.5
  python -m paper_1308_2864_gb300.serve_bench --workload c5 --jobs 512 \
      --rate-fracs 0.25,0.5,0.7,0.9 --maxit 40000 [--precision fp64 --subsample 16]

c4: uneven jobs (N in [20, 48], p = 2 x atoms in [4, 32]) all submitted at
    once; reports solves/s and the latency spread.
    With --mode batch the same jobs run as one job table (ks_batch): every
    kernel launch of an iteration covers all jobs still iterating.
c5: a Poisson stream (N in [24, 96], p in [8, 128]); each arrival rate is a
    fraction of the saturation throughput measured first on the same jobs
    (or --rate jobs/s); --rate-fracs runs one stream per fraction, all with
    the same seeded gaps scaled by the rate.  Reports p50/p99 latency (submit
    to result) and solves/s per stream.  --subsample K runs a seeded K-job
    subsample of the stream instead (for a form too slow for all of it).
Each job runs Alg. ConOptM to ||D||_M <= gtol or --maxit iterations.  One JSON
line per run on stdout.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import threading
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def run(jobs, arrivals, slots, budget, opts):
    """Submit jobs at the given arrival times (s from start, None = at once),
    collect all results; returns (wall s, latencies, results, server stats)."""
    import numpy as np
    import paper_1308_2864_gb300 as ks
    srv = ks.Server(hbm_budget_bytes=budget, max_slots=slots)
    x0 = [np.ascontiguousarray(s.x0()) for s in jobs]
    ids = [None] * len(jobs)
    t0 = time.perf_counter()

    def feeder():
        for i, s in enumerate(jobs):
            if arrivals is not None:
                dt = arrivals[i] - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
            ids[i] = srv.submit(s, x0=x0[i], **opts)

    th = threading.Thread(target=feeder)
    th.start()
    lat, res = [], []
    for i in range(len(jobs)):
        while ids[i] is None:
            time.sleep(1e-4)
        r, _, l = srv.poll(ids[i], wait=True)
        lat.append(l)
        res.append(r)
    th.join()
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    return wall, lat, res, st


def summary(lat, res, wall) -> dict:
    """Throughput and latency of one run: solves/s over its wall time, p50
    and p99 of the submit-to-result latencies, converged jobs."""
    import numpy as np
    return {"solves_per_s": len(lat) / wall, "wall_s": wall,
            "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "converged": sum(r["status"] == 0 for r in res),
            "iters_total": sum(r["iters"] for r in res)}


def serve_streams(jobs, slots, budget, opts, fracs, rate=0.0, seed=1004, run_fn=run):
    """Saturation (all jobs at once), then one Poisson stream per fraction
    of it (or one at `rate` jobs/s when rate > 0).  Returns the saturation
    summary and the list of stream summaries."""
    import ks_inputs as ki
    wall, lat, res, st = run_fn(jobs, None, slots, budget, opts)
    sat = summary(lat, res, wall)
    sat.update({"peak_running": st["peak_running"],
                "peak_gb_in_use": st["peak_bytes_in_use"] / (1 << 30)})
    streams = []
    for frac in ([None] if rate > 0 else fracs):
        r = rate if frac is None else frac * sat["solves_per_s"]
        arr = ki.poisson_arrivals(seed, len(jobs), r)
        wall, lat, res, st = run_fn(jobs, arr, slots, budget, opts)
        row = {"rate_frac": frac, "rate_jobs_per_s": r, **summary(lat, res, wall),
               "peak_running": st["peak_running"]}
        streams.append(row)
    return sat, streams


def main(argv=None) -> int:
    import torch

    import ks_inputs as ki

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="c4", choices=["c4", "c5"])
    ap.add_argument("--jobs", type=int, default=64)
    ap.add_argument("--slots", type=int, default=16)
    ap.add_argument("--budget-gb", type=float, default=180.0)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--maxit", type=int, default=300)
    ap.add_argument("--gtol", type=float, default=1e-6)
    ap.add_argument("--rate", type=float, default=0.0, help="c5 arrivals per second")
    ap.add_argument("--rate-frac", type=float, default=0.5,
                    help="c5: arrival rate as a fraction of the measured saturation throughput")
    ap.add_argument("--rate-fracs", default="",
                    help="c5: comma-separated fractions, one stream each (overrides --rate-frac)")
    ap.add_argument("--subsample", type=int, default=0,
                    help="c5: run a seeded subsample of this many of the --jobs jobs")
    ap.add_argument("--mode", default="server", choices=["server", "batch"],
                    help="c4: continuous-batching server (per-job streams) or one job table")
    ap.add_argument("--fp64-split", type=int, default=0, choices=[0, 1, 2],
                    help="FP64 Grams and updates on the tensor cores by digit splitting")
    ap.add_argument("--no-graphs", action="store_true",
                    help="batch mode: plain launches instead of the captured CUDA graphs")
    ap.add_argument("--autotune", action="store_true",
                    help="batch mode: time and keep the fastest launch shapes first")
    a = ap.parse_args(argv)
    torch.cuda.init()
    jobs = (ki.config_c4_jobs(njobs=a.jobs) if a.workload == "c4"
            else ki.config_c5_jobs(njobs=a.jobs))
    picked = None
    if a.workload == "c5" and 0 < a.subsample < a.jobs:
        picked = ki.stream_subsample(a.subsample, a.jobs)
        jobs = [jobs[i] for i in picked]
    opts = dict(retraction="qr", gtol=a.gtol, maxit=a.maxit, precision=a.precision,
                fp64_split=a.fp64_split)
    budget = int(a.budget_gb * (1 << 30))
    out = {"workload": a.workload, "jobs": a.jobs, "slots": a.slots, "precision": a.precision,
           "maxit": a.maxit, "budget_gb": a.budget_gb, "mode": a.mode, "fp64_split": a.fp64_split,
           "subsample": picked}
    if a.mode == "batch":
        import paper_1308_2864_gb300 as ks
        t0 = time.perf_counter()
        B = ks.Batch(jobs)
        B.set_graphs(not a.no_graphs)
        t_create = time.perf_counter() - t0
        out["graphs"] = not a.no_graphs
        if a.autotune:
            out["autotune"] = B.autotune()
        B.minimize(maxit=2, **{k: v for k, v in opts.items() if k != "maxit"})   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res, _ = B.minimize(**opts)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        out.update({"solves_per_s": a.jobs / wall, "batch_wall_s": wall, "create_s": t_create,
                    "gb": B.bytes / (1 << 30),
                    "converged": sum(r["status"] == 0 for r in res),
                    "iters_total": sum(r["iters"] for r in res),
                    "iters_max": max(r["iters"] for r in res),
                    "ms_per_lockstep_iter": 1e3 * wall / max(1, max(r["iters"] for r in res))})
        print(json.dumps(out), flush=True)
        B.close()
        return 0
    if a.workload == "c4":
        wall, lat, res, st = run(jobs, None, a.slots, budget, opts)
        sat = summary(lat, res, wall)
        out.update({"saturation_solves_per_s": sat["solves_per_s"], "batch_wall_s": wall,
                    "batch_p50_s": sat["p50_latency_s"], "batch_p99_s": sat["p99_latency_s"],
                    "peak_running": st["peak_running"],
                    "peak_gb_in_use": st["peak_bytes_in_use"] / (1 << 30),
                    "converged": sat["converged"], "iters_total": sat["iters_total"]})
        print(json.dumps(out), flush=True)
        return 0
    fracs = ([float(x) for x in a.rate_fracs.split(",") if x.strip()] if a.rate_fracs
             else [a.rate_frac])
    sat, streams = serve_streams(jobs, a.slots, budget, opts, fracs, rate=a.rate)
    out.update({"saturation": sat, "streams": streams})
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
