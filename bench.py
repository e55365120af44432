"""Benchmark: time-to-||grad||_M <= 1e-6 (solves/s) of direct Kohn-Sham
minimisation (Alg. ConOptM, QR retraction) on the 64^3-grid, 32-atom,
p = 64 synthetic system (cube 20 bohr, Z = 4 Gaussian pseudo-atoms on a
jittered 4x4x2 lattice, Slater + PZ81) on one GB300.

One step = one solve from the seeded initial block until ||D||_M <= 1e-6 or
300 iterations (the iteration cap of the 24^3 protocol and of ks_opts), in
the plain FP64 form (value), in the FP32-phase mixed form (config.mixed) and
in FP64 with the Grams and updates on the tensor cores by exact digit
splitting (config.fp64_split).
Prints ONE JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the plain FP64 CPU oracle on the host cores on a
bounded sample of the same workload: W untimed and K timed iterations of the
same solve (one iteration per step), scaled to a 300-iteration solve.  Under torchrun each rank solves its own
replica (no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

METRIC = "time-to-||grad||<=1e-6 & solves/s, p50/p99 latency; mixed vs plain FP64 GPU"
WORKLOAD = "c2: cube 20 bohr, 64^3 Q1 grid, 32 atoms Z=4 jittered 4x4x2 lattice, p=64, Slater+PZ81, QR"
GTOL = 1e-6
MAXIT = 300
# jobs of the batched-jobs recipe (seed 1003) that reach ||D||_M <= 1e-6 in
# a few thousand iterations (1-9 s each)
C4_TTS_JOBS = (1, 2, 4, 5)
# DRAM bytes per launch of the FP64 update kernel: dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture of its projection and retraction
# launches on this workload (mean of the two).  Must be re-measured, or set
# to None, whenever that kernel changes.
COMBINE_FP64_TRAFFIC_BYTES = 3.695e8


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(iters: int = 3, warmup: int = 0):
    """Time the oracle's Alg. ConOptM on the workload, as it stands: its
    one-time set-up (orthonormalisation and the first evaluation), then
    `warmup` untimed and `iters` timed iterations of one solve, each timed
    from the previous iteration's end.  Returns (mean seconds per timed
    iteration, set-up seconds, threads used)."""
    import ks_inputs as ki
    from oracle import energy as oe
    from oracle import stiefel as ost
    s = ki.config_c2()
    model = oe.Model.from_system(s)
    model.vext()
    t0 = time.perf_counter()
    ost.minimize(model, s.x0(), ost.Options(retraction="qr", gtol=GTOL, maxit=0))
    t_setup = time.perf_counter() - t0
    ends = []
    t0 = time.perf_counter()
    ost.minimize(model, s.x0(), ost.Options(retraction="qr", gtol=GTOL, maxit=warmup + iters),
                 callback=lambda k, pt: ends.append(time.perf_counter()))
    # iteration k ends at ends[k]; the first starts once the set-up is done
    spans = np.diff([t0 + t_setup] + ends)
    per_iter = float(np.mean(spans[warmup:warmup + iters]))
    threads = int(os.environ.get("OMP_NUM_THREADS", "0")) or os.cpu_count()
    return per_iter, t_setup, threads


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    iters = MAXIT
    steps = max(args.steps, 1)
    per_iter, t_setup, threads = oracle_sample(steps, args.warmup)
    t_solve = t_setup + per_iter * iters
    value = 1.0 / t_solve
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_solve * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "iterations_assumed": iters,
                   "oracle_seconds_per_iteration": per_iter, "oracle_setup_seconds": t_setup},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "kind": "oracle",
                         "sample": f"{args.warmup} untimed + {steps} timed oracle iterations of "
                                   f"the c2 solve ({per_iter:.2f} s each) + set-up "
                                   f"({t_setup:.1f} s), scaled to a {iters}-iteration solve"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def class_shares(prof) -> dict:
    """Share of each kernel class in the live per-class CUDA-event timings."""
    total = max(sum(v[0] for v in prof.values()), 1e-9)
    return {k: round(v[0] / total, 4) for k, v in prof.items() if v[1] > 0}


def timed_solves(P, X, X0, opts, steps, warmup, stream, barrier, clk=None):
    """W untimed and K timed solves; returns (ms over the K solves, results,
    per-class profile, kernel launches in the timed region)."""
    import torch
    import paper_1308_2864_gb300 as ks

    def solve():
        X.copy_(X0)
        return P.minimize(X, **opts)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            solve()
        stream.synchronize()
        barrier()
        torch.cuda.synchronize()
        launches0 = ks.kernel_launches()
        ks.profile_start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        results = []
        if clk:
            clk.__enter__()
        ev0.record(stream)
        for _ in range(steps):
            results.append(solve())
        ev1.record(stream)
        ev1.synchronize()
        if clk:
            clk.__exit__(None, None, None)
        prof = ks.profile_stop()
        launches = ks.kernel_launches() - launches0
        torch.cuda.synchronize()
        barrier()
    return ev0.elapsed_time(ev1), results, prof, launches


def run_gpu(args):
    import torch
    import ks_inputs as ki
    import paper_1308_2864_gb300 as ks

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(v):
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        if world > 1:
            import torch.distributed as dist
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    s = ki.config_c2()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        P = ks.Problem.from_system(s, stream=stream)
        X0 = torch.from_numpy(np.ascontiguousarray(s.x0())).cuda()
        X = torch.empty_like(X0)
    fp64 = dict(retraction="qr", gtol=GTOL, maxit=MAXIT, precision="fp64")
    mixed = dict(retraction="qr", gtol=GTOL, maxit=MAXIT, precision="mixed")

    clk = ClockSampler(local)
    ms, results, prof, launches = timed_solves(P, X, X0, fp64, args.steps, args.warmup, stream,
                                               barrier, clk)
    ms_max = max_over_ranks(ms)
    value = world * args.steps / (ms_max / 1e3)
    ms_m, res_m, prof_m, _ = timed_solves(P, X, X0, mixed, args.steps, args.warmup, stream, barrier)
    ms_m = max_over_ranks(ms_m)
    # the same FP64 solve with its Grams and updates on the tensor cores by
    # exact digit splitting (ks_set_fp64_emulation 1)
    P.set_fp64_emulation(1)
    ms_s, res_s, prof_s, _ = timed_solves(P, X, X0, fp64, args.steps, args.warmup, stream, barrier)
    ms_s = max_over_ranks(ms_s)
    P.set_fp64_emulation(0)

    # time to ||D||_M <= 1e-6 with and without the split products on a
    # 48-orbital system that converges (14^3 grid, 24 atoms)
    sp = ki.small_system(N=14, L=8.0, natoms=24, p=48, Z=4.0, seed=5)
    sp.rc = 1.0
    split_tts = {}
    for mode in (0, 1):
        with torch.cuda.stream(stream):
            Ps = ks.Problem.from_system(sp, stream=stream)
            Ps.set_fp64_emulation(mode)
            Xs = torch.from_numpy(np.ascontiguousarray(sp.x0())).cuda()
            stream.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rs = Ps.minimize(Xs, gtol=GTOL, maxit=20000)
            e1.record(stream)
            e1.synchronize()
        split_tts["split" if mode else "fp64"] = {
            "seconds": e0.elapsed_time(e1) / 1e3, "iters": rs["iters"], "energy": rs["E"],
            "converged": rs["status"] == 0}
        Ps.close()
    split_tts["energy_difference_Ha"] = split_tts["split"]["energy"] - split_tts["fp64"]["energy"]
    split_tts["system"] = "14^3 grid, 24 atoms (Z=4, rc=1), p=48, QR, to ||D||_M <= 1e-6"

    # time to ||D||_M <= 1e-6 on the 24^3 two-atom system (it converges in
    # ~1300 iterations): plain FP64 against the FP32 phase + FP64 polish
    c1 = ki.config_c1()
    with torch.cuda.stream(stream):
        P1 = ks.Problem.from_system(c1, stream=stream)
        X1 = torch.from_numpy(np.ascontiguousarray(c1.x0())).cuda()
        Y1 = torch.empty_like(X1)
    c1_out = {}
    for prec in ("fp64", "mixed"):
        o = dict(retraction="cayley", gtol=GTOL, maxit=20000, precision=prec)
        with torch.cuda.stream(stream):
            Y1.copy_(X1)
            P1.minimize(Y1, **o)                      # warm-up
            Y1.copy_(X1)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            r1 = P1.minimize(Y1, **o)
            ev1.record(stream)
            ev1.synchronize()
        sec = ev0.elapsed_time(ev1) / 1e3
        c1_out[prec] = {"seconds": sec, "iters": r1["iters"],
                        "us_per_iteration": 1e6 * sec / max(r1["iters"], 1),
                        "cg_iters_total": r1["cg_iters_total"], "backtracks": r1["backtracks"],
                        "fp32_phase_iters": r1["mixed_iters"], "gradnorm": r1["gradnorm"],
                        "energy": r1["E"], "converged": r1["status"] == 0}
    c1_out["energy_difference_Ha"] = c1_out["mixed"]["energy"] - c1_out["fp64"]["energy"]
    P1.close()

    # time to ||D||_M <= 1e-6 on converging systems of the batched-jobs
    # recipe (grids 24^3..38^3, p = 26..32): plain FP64 against the mixed form
    c4_out = {"jobs": [], "fp64_s": 0.0, "mixed_s": 0.0}
    c4_jobs = ki.config_c4_jobs(njobs=8)
    for j in C4_TTS_JOBS:
        sj = c4_jobs[j]
        with torch.cuda.stream(stream):
            Pj = ks.Problem.from_system(sj, stream=stream)
            Xj0 = torch.from_numpy(np.ascontiguousarray(sj.x0())).cuda()
            Yj = torch.empty_like(Xj0)
        row = {"job": j, "N": sj.N, "p": sj.p}
        for prec in ("fp64", "mixed"):
            o = dict(retraction="qr", gtol=GTOL, maxit=20000, precision=prec)
            with torch.cuda.stream(stream):
                Yj.copy_(Xj0)
                Pj.minimize(Yj, **{**o, "maxit": 3})         # warm-up
                Yj.copy_(Xj0)
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                rj = Pj.minimize(Yj, **o)
                ev1.record(stream)
                ev1.synchronize()
            secs = ev0.elapsed_time(ev1) / 1e3
            row[prec] = {"seconds": secs, "iters": rj["iters"], "energy": rj["E"],
                         "converged": rj["status"] == 0, "fp32_phase_iters": rj["mixed_iters"]}
            c4_out[prec + "_s"] += secs
        row["energy_difference_Ha"] = row["mixed"]["energy"] - row["fp64"]["energy"]
        c4_out["jobs"].append(row)
        Pj.close()
    c4_out["speedup"] = c4_out["fp64_s"] / max(c4_out["mixed_s"], 1e-12)

    # end to end through the host entry point: X0 from pinned host memory in,
    # the final block back out, every step
    x0_np = s.x0()
    Xh = torch.from_numpy(np.ascontiguousarray(x0_np)).pin_memory()
    Xh_np = Xh.numpy()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        np.copyto(Xh_np, x0_np)
        P.minimize_host(Xh_np, **fp64)
    torch.cuda.synchronize()
    e2e_value = world * e2e_steps / max_over_ranks(time.perf_counter() - t0)
    nbytes = s.n * s.p * 8

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel class from the live CUDA-event timings
    # and the library's algorithmic work counts
    total_ms = sum(v[0] for v in prof.values())
    name, (dms, dcnt, dfl, dby) = max(prof.items(), key=lambda kv: kv[1][0])
    shares = {k: round(v[0] / total_ms, 4) for k, v in prof.items() if v[1] > 0}
    fp64_peak = 152 * 4 * 2.07e9 / 1e12       # TFLOP/s: 2 DFMA/clk/SM at 2070 MHz
    achieved = dfl / (dms / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": achieved / fp64_peak,
            "traffic": COMBINE_FP64_TRAFFIC_BYTES if name == "combine" else None,
            "kernel": f"{name} (FP64)", "launches": dcnt,
            "peak_note": "FP64 FMA peak derived from 152 SMs x 4 flop/clk x 2.07 GHz "
                         "(probe measured 1.20 TFLOP/s at 1.99 GHz)"}
    r0 = results[-1]
    rm = res_m[-1]
    per_iter, t_setup, threads = oracle_sample(3)
    cpu_value = 1.0 / (t_setup + per_iter * max(r0["iters"], 1))
    per_solve = [r["seconds"] for r in results]
    mixed_kernel = class_shares(prof_m)
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "fp64", "retraction": "qr", "gtol": GTOL,
                   "maxit": MAXIT, "iters_per_solve": r0["iters"],
                   "converged": r0["status"] == 0, "final_gradnorm": r0["gradnorm"],
                   "final_energy": r0["E"], "ms_per_iteration": ms_max / args.steps / max(r0["iters"], 1),
                   "cg_iters_per_solve": r0["cg_iters_total"],
                   "p50_s": statistics.median(per_solve),
                   "p99_s": float(np.percentile(per_solve, 99)),
                   "l2": "working set ~1.7 GB > 129 MB L2 (no flush needed)",
                   "parallelism": f"replicas x{world}",
                   "mixed": {"solves_per_s": world * args.steps / (ms_m / 1e3),
                             "ms_per_step": ms_m / args.steps, "iters_per_solve": rm["iters"],
                             "fp32_phase_iters": rm["mixed_iters"],
                             "final_gradnorm": rm["gradnorm"], "final_energy": rm["E"],
                             "energy_minus_fp64_Ha": rm["E"] - r0["E"],
                             "kernel_shares": mixed_kernel},
                   "fp64_split": {"solves_per_s": world * args.steps / (ms_s / 1e3),
                                  "ms_per_step": ms_s / args.steps,
                                  "ms_per_iteration": ms_s / args.steps / max(res_s[0]["iters"], 1),
                                  "iters_per_solve": res_s[0]["iters"],
                                  "final_gradnorm": res_s[0]["gradnorm"],
                                  "final_energy": res_s[0]["E"],
                                  "energy_minus_fp64_Ha": res_s[0]["E"] - r0["E"],
                                  "kernel_shares": class_shares(prof_s),
                                  "note": "Grams and updates as BF16 tcgen05 MMAs of exact digit "
                                          "splits (48/56 bits per operand), folded in int64 "
                                          "before one FP64 rounding",
                                  "time_to_solution": split_tts},
                   "c1_time_to_solution": c1_out,
                   "c4_time_to_solution": c4_out},
        "roofline": roof,
        "kernel_shares": shares,
        "cpu_baseline": {"value": cpu_value, "unit": "solves/s", "cores": threads, "kind": "oracle",
                         "sample": f"3 oracle iterations of the same solve ({per_iter:.2f} s each) "
                                   f"+ set-up {t_setup:.2f} s, scaled to {r0['iters']} iterations"},
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
