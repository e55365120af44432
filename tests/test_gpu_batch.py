"""Batched job table (ks_batch): per-job results against the single-system
path and the FP64 oracle, independence of a job's result from its batch
mates, the mixed-precision batch, and argument checks."""
import numpy as np
import pytest

import ks_inputs as ki
from oracle import energy as oe
from oracle import stiefel as ost

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def easy(N, natoms, p, Z, seed, L=7.0):
    # resolved pseudo-atoms (rc = 1): converge in a few hundred iterations
    s = ki.small_system(N=N, L=L, natoms=natoms, p=p, Z=Z, seed=seed)
    s.rc = 1.0
    return s


def harder():
    # p = 10 (tiled Gram, narrow update, PC = 8) and p = 36 (tiled update,
    # PC = 32) with c4-like pseudo-atoms (Z = 4, p = 2 atoms)
    return [ki.small_system(N=13, L=7.0, natoms=5, p=10, seed=5),
            ki.small_system(N=11, L=8.0, natoms=18, p=36, seed=6)]


def single(s, **kw):
    import paper_1308_2864_gb300 as ks
    P = ks.Problem.from_system(s)
    X = torch.from_numpy(np.ascontiguousarray(s.x0())).cuda()
    r = P.minimize(X, **kw)
    return r, X.cpu().numpy()


def test_batch_converges_to_single_path_and_oracle():
    import paper_1308_2864_gb300 as ks
    jobs = [easy(10, 2, 2, 1.0, 7), easy(12, 2, 4, 2.0, 8), easy(9, 1, 1, 2.0, 3, L=6.0)]
    B = ks.Batch(jobs)
    res, Xs = B.minimize(retraction="qr", gtol=1e-8, maxit=3000)
    for s, r, X in zip(jobs, res, Xs):
        assert r["status"] == 0 and r["gradnorm"] <= 1e-8
        rs, _ = single(s, retraction="qr", gtol=1e-8, maxit=3000)
        assert r["E"] == pytest.approx(rs["E"], abs=1e-8)
        model = oe.Model.from_system(s)
        assert ost.ortho_error(model, X) < 1e-12
        # the energy of the returned block, recomputed by the oracle
        assert oe.evaluate(model, X).E == pytest.approx(r["E"], abs=1e-9)
    ref = ost.minimize(oe.Model.from_system(jobs[0]), jobs[0].x0(),
                       ost.Options(retraction="qr", gtol=1e-8, maxit=2000))
    assert res[0]["E"] == pytest.approx(ref.E, abs=1e-8)


def test_batch_early_iterations_match_single_path():
    # uneven sizes across the stencil, Gram and update variants: after a
    # few iterations every job sits where the single-system path is
    import paper_1308_2864_gb300 as ks
    jobs = [easy(10, 2, 2, 1.0, 7)] + harder()
    B = ks.Batch(jobs)
    res, Xs = B.minimize(retraction="qr", gtol=1e-12, maxit=12)
    for s, r, X in zip(jobs, res, Xs):
        assert r["iters"] == 12
        rs, Xd = single(s, retraction="qr", gtol=1e-12, maxit=12)
        assert r["E"] == pytest.approx(rs["E"], rel=1e-9)
        assert np.abs(X - Xd).max() <= 1e-6 * np.abs(Xd).max()


def test_batch_result_does_not_depend_on_batch_mates():
    import paper_1308_2864_gb300 as ks
    a = easy(10, 2, 2, 1.0, 7)
    alone, Xa = ks.Batch([a]).minimize(retraction="qr", gtol=1e-12, maxit=20)
    mixed_in, Xm = ks.Batch(harder() + [a]).minimize(retraction="qr", gtol=1e-12, maxit=20)
    assert alone[0]["E"] == mixed_in[-1]["E"]
    assert np.array_equal(Xa[0], Xm[-1])


def test_batch_mixed_precision_then_polish():
    import paper_1308_2864_gb300 as ks
    jobs = [easy(10, 2, 2, 1.0, 7), easy(12, 2, 4, 2.0, 8)]
    r64, _ = ks.Batch(jobs).minimize(retraction="qr", gtol=1e-8, maxit=3000)
    rmx, Xs = ks.Batch(jobs).minimize(retraction="qr", gtol=1e-8, maxit=3000,
                                      precision="mixed", polish_gtol=1e-4)
    for s, a, b, X in zip(jobs, r64, rmx, Xs):
        assert b["status"] == 0 and b["gradnorm"] <= 1e-8
        assert b["mixed_iters"] > 0
        assert b["E"] == pytest.approx(a["E"], abs=1e-8)
        assert ost.ortho_error(oe.Model.from_system(s), X) < 1e-12


def test_batch_rejects_what_it_does_not_support():
    import paper_1308_2864_gb300 as ks
    with pytest.raises(ks.KSError):
        ks.Batch([ki.small_system(N=6, L=6.0, natoms=2, p=105, seed=1)])
    B = ks.Batch([easy(10, 2, 2, 1.0, 7)])
    with pytest.raises(ks.KSError):
        B.minimize(retraction="cayley", maxit=5)


def test_batch_graphs_and_plain_launches_agree():
    # the captured step sequences replay exactly the plain launches
    import paper_1308_2864_gb300 as ks
    jobs = [easy(10, 2, 2, 1.0, 7)] + harder()
    out = []
    for g in (True, False):
        B = ks.Batch(jobs)
        B.set_graphs(g)
        out.append(B.minimize(retraction="qr", gtol=1e-12, maxit=15, precision="mixed",
                              polish_gtol=1e-3))
    for a, b, xa, xb in zip(out[0][0], out[1][0], out[0][1], out[1][1]):
        assert a["E"] == b["E"] and a["iters"] == b["iters"]
        assert np.array_equal(xa, xb)


def test_batch_autotune_keeps_results_up_to_summation_order():
    import paper_1308_2864_gb300 as ks
    jobs = [easy(10, 2, 2, 1.0, 7)] + harder()
    ref, Xr = ks.Batch(jobs).minimize(retraction="qr", gtol=1e-12, maxit=12)
    B = ks.Batch(jobs)
    choice = B.autotune()
    assert choice["gram_rows"] in (1024, 2048, 4096, 8192, 16384)
    assert choice["comb_per_thread"] in (2, 4, 8, 16)
    assert choice["pot_per_thread"] in (1, 2, 4, 8)
    assert choice["stencil_planes"] in (0, 8, 16, 32, 64)
    res, Xs = B.minimize(retraction="qr", gtol=1e-12, maxit=12)
    for a, b, xa, xb in zip(ref, res, Xr, Xs):
        assert b["status"] == a["status"] and b["iters"] == a["iters"]
        assert b["E"] == pytest.approx(a["E"], rel=1e-10)
        assert np.abs(xb - xa).max() <= 1e-7 * np.abs(xa).max()
