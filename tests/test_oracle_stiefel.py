"""Pins of the oracle's manifold optimiser: projected gradient (Eq.
def-nablaE), Cholesky-QR retraction (Eq. QR, Alg. ChQR, Prop. 3.1), Cayley
retraction (Lemma 3.1: Eqs. WY1, WY3, WY-1d), the nonmonotone search
(Eq. NMLS-Armijo) and Alg. ConOptM against closed forms and brute force."""
import math

import numpy as np
import pytest
from scipy.linalg import eigh

import ks_inputs as ki
from oracle import brute, energy, fe, stiefel


def _model(N=5, L=5.0, natoms=2, p=3, Z=2.0, seed=5, rc=1.0, **kw):
    s = ki.small_system(N=N, L=L, natoms=natoms, p=p, Z=Z, seed=seed)
    s.rc = rc
    return energy.Model.from_system(s, **kw), s


def _feasible_point(model, s):
    X = stiefel.m_orthonormalize(model, s.x0())
    return stiefel.point_at(model, X)


def test_m_orthonormalize():
    model, s = _model()
    X = stiefel.m_orthonormalize(model, s.x0())
    assert stiefel.ortho_error(model, X) < 1e-13


def test_gradient_is_tangent_and_matches_y_coordinates():
    from scipy.linalg import sqrtm
    model, s = _model(N=4)
    pt = _feasible_point(model, s)
    XtMD = pt.X.T @ pt.MD
    assert np.abs(XtMD + XtMD.T).max() < 1e-12                 # tangent at X
    # Eq. def-nablaE in Y = M^{1/2} X coordinates, mapped back
    _, M = fe.dense_K_M(model.N, model.h)
    Mh = np.real(sqrtm(M))
    Y = Mh @ pt.X
    EY = np.linalg.solve(Mh, pt.ev.EX)
    gradY = EY - Y @ EY.T @ Y
    assert np.allclose(np.linalg.solve(Mh, gradY), pt.D, atol=1e-11)
    assert pt.dnorm2 == pytest.approx(float(np.sum(gradY * gradY)), rel=1e-10)


def test_gradient_vanishes_on_exact_eigenspace():
    # V = 0: the minimiser is spanned by the lowest generalised eigenvectors.
    model, s = _model(N=5, p=4, use_ext=False, use_hartree=False, use_xc=False)
    K, M = fe.dense_K_M(model.N, model.h)
    w, V = eigh(K, M, subset_by_index=[0, 3])
    pt = stiefel.point_at(model, V)
    assert pt.dnorm < 1e-11


@pytest.mark.parametrize("tau", [0.0, 0.05, 0.7])
def test_qr_retraction_prop31(tau):
    model, s = _model()
    pt = _feasible_point(model, s)
    Y = pt.X - tau * pt.D
    YMY = Y.T @ fe.apply_M(Y, model.N, model.h)
    DMD = pt.D.T @ pt.MD
    # Prop. 3.1 in the M metric: Y^T M Y = I + tau^2 D^T M D ...
    assert np.allclose(YMY, np.eye(model.p) + tau * tau * DMD, atol=1e-12)
    lam = np.linalg.eigvalsh(YMY)
    nrm2 = np.linalg.eigvalsh(DMD).max()
    # ... so 1 <= lambda(Y^T M Y) <= 1 + tau^2 ||D||_2^2
    assert lam.min() >= 1 - 1e-12 and lam.max() <= 1 + tau * tau * nrm2 + 1e-12
    Xn = stiefel.retract_qr(model, pt, tau)
    assert stiefel.ortho_error(model, Xn) < 1e-12
    if tau == 0.0:
        assert np.allclose(Xn, pt.X, atol=1e-13)               # R(0) = X


@pytest.mark.parametrize("retract", [stiefel.retract_qr, stiefel.retract_cayley])
def test_retraction_derivative_is_minus_gradient(retract):
    model, s = _model()
    pt = _feasible_point(model, s)
    t = 1e-6
    dXdt = (retract(model, pt, t) - retract(model, pt, -t)) / (2 * t)
    assert np.allclose(dXdt, -pt.D, atol=1e-7 * np.abs(pt.D).max())


def test_cayley_woodbury_equals_dense_and_preserves_metric():
    model, s = _model(N=4, p=3)
    pt = _feasible_point(model, s)
    for tau in (0.01, 0.3, 2.0):
        X3 = stiefel.retract_cayley(model, pt, tau)
        X1 = stiefel.retract_cayley_dense(model, pt, tau)
        assert np.allclose(X3, X1, atol=1e-11)
        M = fe.apply_M(X3, model.N, model.h)
        assert np.allclose(X3.T @ M, pt.X.T @ pt.MX, atol=1e-12)


def test_cayley_p1_closed_form():
    model, s = _model(N=4, p=1, natoms=1, Z=2.0)
    pt = _feasible_point(model, s)
    for tau in (0.02, 0.5, 3.0):
        assert np.allclose(stiefel.retract_cayley_p1(model, pt, tau),
                           stiefel.retract_cayley(model, pt, tau), atol=1e-12)
        assert np.allclose(stiefel.retract_cayley_p1(model, pt, tau),
                           stiefel.retract_cayley_dense(model, pt, tau), atol=1e-11)


def test_bb_step_rules():
    opt = stiefel.Options()
    assert stiefel.bb_step(1, 2.0, -4.0, 9.0, opt) == pytest.approx(0.5)      # ss/|sy|
    assert stiefel.bb_step(2, 2.0, -4.0, 8.0, opt) == pytest.approx(0.5)      # |sy|/yy
    assert stiefel.bb_step(1, 1.0, 0.0, 1.0, opt) == opt.tau0
    assert stiefel.bb_step(2, 1.0, 1.0, float("nan"), opt) == opt.tau0
    assert stiefel.bb_step(1, 1e30, 1.0, 1.0, opt) == opt.tau_max


@pytest.mark.parametrize("retraction", ["qr", "cayley"])
def test_minimize_v0_closed_form(retraction):
    # Non-interacting, V = 0: E* = (f/2) * sum of the p lowest generalised
    # eigenvalues of (K, M); p = 4 closes the (1,1,1) + 3 x (2,1,1) shell.
    model, s = _model(N=6, L=6.0, p=4, use_ext=False, use_hartree=False, use_xc=False)
    lam = fe.generalized_eigs_closed_form(model.N, model.h)
    want = 0.5 * model.occ * lam[:4].sum()
    r = stiefel.minimize(model, s.x0(), stiefel.Options(retraction=retraction, gtol=1e-8, maxit=2000))
    assert r.converged
    assert r.E == pytest.approx(want, abs=1e-10)
    assert stiefel.ortho_error(model, r.X) < 1e-12


def test_minimize_external_only_dense_eigensolve():
    model, s = _model(N=6, L=6.0, p=3, natoms=2, Z=3.0, use_hartree=False, use_xc=False)
    K, M = fe.dense_K_M(model.N, model.h)
    H = 0.5 * K + model.h ** 3 * np.diag(model.vext())
    w = eigh(H, M, eigvals_only=True, subset_by_index=[0, 2])
    want = model.occ * w.sum() + model.eii()
    r = stiefel.minimize(model, s.x0(), stiefel.Options(gtol=1e-8, maxit=3000))
    assert r.converged
    assert r.E == pytest.approx(want, abs=1e-10)


@pytest.mark.parametrize("case", [
    dict(N=7, L=6.0, natoms=1, p=1, Z=2.0, seed=7),
    dict(N=7, L=7.0, natoms=2, p=2, Z=1.0, seed=7),
])
@pytest.mark.parametrize("retraction", ["qr", "cayley"])
def test_minimize_interacting_matches_scf(case, retraction):
    model, s = _model(rc=1.0, **case)
    E_scf, X_scf, w = brute.scf_reference(model)
    r = stiefel.minimize(model, s.x0(), stiefel.Options(retraction=retraction, gtol=1e-9, maxit=3000))
    assert r.converged
    assert r.E == pytest.approx(E_scf, abs=1e-10)
    # KKT (Eq. disKS with the mass metric): H X = M X Lambda, Lambda symmetric
    H = brute.hamiltonian_dense(model, energy.density(r.X, model.occ))
    Lam = r.X.T @ H @ r.X
    assert np.abs(Lam - Lam.T).max() < 1e-8
    _, M = fe.dense_K_M(model.N, model.h)
    assert np.abs(H @ r.X - M @ r.X @ Lam).max() < 1e-7
    assert np.allclose(np.sort(np.linalg.eigvalsh(0.5 * (Lam + Lam.T))), w, atol=1e-8)


def test_nonmonotone_reference_decreases_and_armijo_holds():
    model, s = _model(N=6, L=6.0, natoms=2, p=2, Z=2.0)
    opt = stiefel.Options(gtol=1e-8, maxit=400)
    r = stiefel.minimize(model, s.x0(), opt)
    prevC = None
    for h in r.history:
        if prevC is not None:
            assert h["C"] <= prevC + 1e-12
        prevC = h["C"]
    assert r.converged and r.dnorm <= 1e-8
    assert all(h["h"] < opt.max_backtrack for h in r.history)


def test_forced_acceptance_restarts_the_reference():
    # With no backtracking allowed and a first step far too long, trials are
    # taken without meeting the Armijo test; each restarts the nonmonotone
    # reference at its energy, so C_k >= E_k holds at every iteration (a
    # reference left below the energy would reject every later step).
    model, s = _model(N=6, L=6.0, natoms=2, p=2, Z=2.0)
    opt = stiefel.Options(gtol=1e-8, maxit=60, max_backtrack=0, tau0=5.0)
    r = stiefel.minimize(model, s.x0(), opt)
    forced = [h for h in r.history if h["forced"]]
    assert forced, "the long first step should fail the test"
    for h in forced:
        assert h["C"] == h["E"] and h["Q"] == 1.0
    assert all(h["C"] >= h["E"] - 1e-12 * abs(h["E"]) for h in r.history)



def test_armijo_rounding_slack_stays_within_its_bound():
    # The rounding slack of the FP64 line search (accept a rise of at most
    # 4 eps sum |E_parts| above the Armijo bound of Eq. NMLS-Armijo): with it
    # on, no unforced step exceeds the exact test's bound by more than the
    # slack, and the run reaches the same minimiser as the exact test, deep
    # into the regime where the required decrease is below the rounding of E.
    model, s = _model(N=6, L=6.0, natoms=2, p=2, Z=2.0)
    exact = stiefel.minimize(model, s.x0(), stiefel.Options(gtol=1e-9, maxit=600))
    opt = stiefel.Options(gtol=1e-9, maxit=600, armijo_slack=True)
    slack = stiefel.minimize(model, s.x0(), opt)
    assert exact.converged and slack.converged
    eps = 2.220446049250313e-16
    for h in slack.history:
        assert 0.0 < h["slack"] < 1e-12
        if not h["forced"]:
            assert h["excess"] <= h["slack"]
    assert slack.E == pytest.approx(exact.E, abs=1e-11)
    assert all(h["excess"] <= 0.0 or h["forced"] for h in exact.history)
    # and the bound is the stated one: recompute it from a trial's parts
    pt = _feasible_point(model, s)
    assert stiefel.armijo_slack(pt.ev.parts, opt) == pytest.approx(
        4.0 * eps * sum(abs(v) for v in pt.ev.parts.values()), rel=1e-15)
    assert stiefel.armijo_slack(pt.ev.parts, stiefel.Options()) == 0.0
