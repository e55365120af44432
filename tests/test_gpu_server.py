"""Serving loop with continuous batching (ks_server_*): results are bitwise
the same alone and in the mix, admission respects the HBM budget and the
slot count, and over-budget jobs are refused at submission."""
import numpy as np
import pytest

import ks_inputs as ki

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OPTS = dict(retraction="qr", gtol=1e-6, maxit=40)


def _jobs():
    return [ki.small_system(N=N, L=0.4 * (N + 1), natoms=a, p=2 * a, Z=4.0, seed=100 + j)
            for j, (N, a) in enumerate([(12, 1), (16, 2), (14, 3), (20, 2), (10, 1), (18, 4)])]


def _alone(s, **opts):
    import paper_1308_2864_gb300 as ks
    P = ks.Problem.from_system(s)
    X = torch.from_numpy(np.ascontiguousarray(s.x0())).cuda()
    r = P.minimize(X, **opts)
    return r, X.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_results_identical_alone_and_in_the_mix(precision):
    import paper_1308_2864_gb300 as ks
    jobs = _jobs()
    srv = ks.Server(hbm_budget_bytes=8 << 30, max_slots=4)
    ids = [srv.submit(s, precision=precision, **OPTS) for s in jobs]
    got = [srv.poll(i, wait=True, want_x=True, n=s.n, p=s.p) for i, s in zip(ids, jobs)]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(jobs) and st["peak_running"] >= 2
    for s, (r, X, lat) in zip(jobs, got):
        ra, Xa = _alone(s, precision=precision, **OPTS)
        assert r["E"] == ra["E"] and r["iters"] == ra["iters"]
        assert np.array_equal(X, Xa)
        assert lat > 0


def test_admission_respects_budget_and_slots():
    import paper_1308_2864_gb300 as ks
    jobs = _jobs()
    sizes = [ks.Problem.bytes_for(s.N, s.p) + s.n * s.p * 8 for s in jobs]
    budget = int(sorted(sizes)[-1] + sorted(sizes)[-2])   # the two largest fit together
    srv = ks.Server(hbm_budget_bytes=budget, max_slots=3)
    ids = [srv.submit(s, **OPTS) for s in jobs]
    for i in ids:
        assert srv.poll(i, wait=True) is not None
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(jobs)
    assert 0 < st["peak_bytes_in_use"] <= budget
    assert st["peak_running"] <= 3


def test_over_budget_job_is_refused():
    import paper_1308_2864_gb300 as ks
    s = _jobs()[0]
    srv = ks.Server(hbm_budget_bytes=1 << 20, max_slots=1)
    with pytest.raises(ks.KSError) as e:
        srv.submit(s, **OPTS)
    assert e.value.status == ks.KS_ENOMEM
    srv.close()


def test_poll_without_wait_reports_running_jobs():
    import paper_1308_2864_gb300 as ks
    s = ki.config_c1()
    srv = ks.Server(hbm_budget_bytes=8 << 30, max_slots=1)
    a = srv.submit(s, retraction="cayley", maxit=300)
    b = srv.submit(s, retraction="cayley", maxit=5)
    assert srv.poll(b, wait=False) is None          # queued behind a
    ra = srv.poll(a, wait=True)
    rb = srv.poll(b, wait=True)
    srv.close()
    assert ra[0]["iters"] == 300 and rb[0]["iters"] == 5


def test_concurrent_polls_of_one_job():
    # two threads wait on the same id: one collects the job, the other is
    # told it is gone (never a wait on a job another poll has freed)
    import threading
    import paper_1308_2864_gb300 as ks
    s = ki.config_c1()
    srv = ks.Server(hbm_budget_bytes=8 << 30, max_slots=1)
    jid = srv.submit(s, retraction="cayley", maxit=200)
    out = [None, None]

    def poll(i):
        try:
            out[i] = srv.poll(jid, wait=True)
        except ks.KSError as e:
            out[i] = e

    ts = [threading.Thread(target=poll, args=(i,)) for i in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=300)
    alive = any(t.is_alive() for t in ts)
    srv.close()
    assert not alive
    got = [o for o in out if isinstance(o, tuple)]
    gone = [o for o in out if isinstance(o, ks.KSError)]
    assert len(got) == 1 and len(gone) == 1
    assert got[0][0]["iters"] == 200 and gone[0].status == ks.KS_EINVAL
