"""Parity of uniform refinement (Alg. AdpConOptM with every element refined)
with the oracle: the Q1 prolongation kernel entry by entry, and the
continuation driver's levels against the oracle's on the same inputs."""
import numpy as np
import pytest

import ks_inputs as ki
from oracle import energy as oe
from oracle import fe as ofe
from oracle import stiefel as ost

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("Nc,p", [(5, 3), (13, 1), (31, 64), (2, 70)])
def test_prolong_matches_oracle(Nc, p):
    # every weight is 1 or 1/2 and both sides nest the sums z, y, x, so the
    # FP64 results agree bit for bit; FP32 within one rounding of the FP64 value
    import paper_1308_2864_gb300 as ks
    rng = np.random.default_rng(Nc * 100 + p)
    Xc = rng.standard_normal((Nc ** 3, p))
    want = ofe.prolong(Xc, Nc)
    got = ks.prolong(dev(Xc), Nc).cpu().numpy()
    assert np.array_equal(got, want)
    got32 = ks.prolong(dev(Xc, torch.float32), Nc).cpu().numpy().astype(np.float64)
    want32 = ofe.prolong(Xc.astype(np.float32).astype(np.float64), Nc)
    assert np.abs(got32 - want32).max() <= 2.0 ** -23 * np.abs(want32).max() * 2


def test_prolong_rejects_bad_arguments():
    import paper_1308_2864_gb300 as ks
    lib = ks.load_library()
    buf = torch.zeros(4096, dtype=torch.float64, device="cuda")
    assert lib.ks_prolong(0, 1, buf.data_ptr(), buf.data_ptr() + 8 * 2048, None) == ks.KS_EINVAL
    assert lib.ks_prolong(2, 1, buf.data_ptr(), buf.data_ptr() + 8, None) == ks.KS_EINVAL  # overlap
    assert lib.ks_prolong(2, 0, buf.data_ptr(), buf.data_ptr() + 8 * 2048, None) == ks.KS_EINVAL


@pytest.mark.parametrize("kind,N,levels", [("ks", 11, 2), ("of", 11, 2), ("ks", 15, 3)])
def test_minimize_refine_matches_oracle(kind, N, levels):
    import paper_1308_2864_gb300 as ks
    if kind == "ks":
        s = ki.small_system(N=N, L=7.0, natoms=2, p=2, Z=1.0, seed=7)
        s.rc = 1.0
    else:
        s = ki.small_of_system(N=N, L=7.0, natoms=2, Z=1.0, seed=11)
    model = oe.Model.from_system(s)
    grids = ost.refine_levels(N, levels)
    x0 = s.x0_for(grids[0])
    opt = ost.Options(retraction="qr", gtol=1e-8, maxit=3000)
    ref = ost.minimize_refine(model, x0, levels, opt, coarse_gtol=1e-3)
    res, X = ks.minimize_refine(s, levels, x0=x0, coarse_gtol=1e-3, retraction="qr", gtol=1e-8,
                                maxit=3000)
    assert len(res) == levels
    for r, o in zip(res[:-1], ref[:-1]):
        assert r["status"] == 0 and r["gradnorm"] <= 1e-3
        assert r["E"] == pytest.approx(o.E, abs=1e-5)
    assert res[-1]["status"] == 0 and res[-1]["gradnorm"] <= 1e-8
    assert res[-1]["E"] == pytest.approx(ref[-1].E, abs=1e-8)
    assert ost.ortho_error(model, X) < 1e-12
    # the same minimiser as a cold single-grid run
    direct = ost.minimize(model, s.x0(), opt)
    assert res[-1]["E"] == pytest.approx(direct.E, abs=1e-8)


def test_minimize_refine_rejects_bad_levels():
    import paper_1308_2864_gb300 as ks
    s = ki.small_system(N=12, L=7.0, natoms=1, p=1)
    with pytest.raises(ks.KSError):
        ks.minimize_refine(s, 2, x0=np.zeros((125, 1)))       # 13 is odd
