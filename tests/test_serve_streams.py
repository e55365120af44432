"""Host logic of the served-stream runner (serving-stream recipe: Poisson
arrivals at fractions of the saturation throughput, p50/p99 latency): the
seeded job subsample, the per-fraction streams and their summaries, with a
stand-in for the server run (no GPU)."""
import numpy as np

import ks_inputs as ki
from paper_1308_2864_gb300 import serve_bench as sb


def test_stream_subsample_is_seeded_distinct_and_sorted():
    a = ki.stream_subsample(16)
    assert a == ki.stream_subsample(16)
    assert len(a) == 16 and len(set(a)) == 16 and a == sorted(a)
    assert 0 <= a[0] and a[-1] < 512
    assert a != ki.stream_subsample(16, seed=7)
    assert ki.stream_subsample(600) == list(range(512))
    assert ki.stream_subsample(0) == []
    # a Fisher-Yates prefix: every index is about equally likely over seeds
    hits = np.zeros(512)
    for seed in range(400):
        hits[ki.stream_subsample(16, seed=seed)] += 1
    assert hits.sum() == 400 * 16 and hits.max() < 40


def test_summary_percentiles_and_counts():
    lat = list(np.arange(1, 101, dtype=float))
    res = [{"status": 0 if i % 4 else 4, "iters": 10} for i in range(100)]
    out = sb.summary(lat, res, wall=20.0)
    assert out["solves_per_s"] == 5.0 and out["wall_s"] == 20.0
    assert out["p50_latency_s"] == np.percentile(lat, 50)
    assert out["p99_latency_s"] == np.percentile(lat, 99)
    assert out["converged"] == 75 and out["iters_total"] == 1000


def _fake_run(calls):
    # every job takes 0.5 s of service; all at once they finish in 4 s
    def run(jobs, arrivals, slots, budget, opts):
        calls.append(arrivals)
        n = len(jobs)
        if arrivals is None:
            return 4.0, [0.5 + 3.5 * i / n for i in range(n)], [{"status": 0, "iters": 5}] * n, \
                {"peak_running": slots, "peak_bytes_in_use": 2 << 30}
        wall = float(arrivals[-1]) + 0.5
        return wall, [0.5] * n, [{"status": 0, "iters": 5}] * n, \
            {"peak_running": 3, "peak_bytes_in_use": 1 << 30}
    return run


def test_streams_at_fractions_of_saturation():
    jobs = list(range(40))
    calls = []
    sat, streams = sb.serve_streams(jobs, 8, 1 << 34, {}, [0.25, 0.5, 0.7, 0.9],
                                    run_fn=_fake_run(calls))
    assert sat["solves_per_s"] == 10.0 and sat["peak_running"] == 8
    assert sat["peak_gb_in_use"] == 2.0
    assert [s["rate_frac"] for s in streams] == [0.25, 0.5, 0.7, 0.9]
    assert [s["rate_jobs_per_s"] for s in streams] == [2.5, 5.0, 7.0, 9.0]
    # one saturation run, then one stream per fraction, with the same
    # seeded gaps scaled by 1 / rate
    assert calls[0] is None and len(calls) == 5
    base = ki.poisson_arrivals(1004, 40, 1.0)
    for arr, s in zip(calls[1:], streams):
        np.testing.assert_allclose(arr * s["rate_jobs_per_s"], base, rtol=1e-12)
        assert s["p50_latency_s"] == 0.5 and s["converged"] == 40


def test_stream_at_a_fixed_rate():
    calls = []
    sat, streams = sb.serve_streams(list(range(10)), 4, 1 << 34, {}, [0.5], rate=3.0,
                                    run_fn=_fake_run(calls))
    assert len(streams) == 1 and streams[0]["rate_frac"] is None
    assert streams[0]["rate_jobs_per_s"] == 3.0
