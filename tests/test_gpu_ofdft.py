"""Parity of the orbital-free path (Sec. 2.2, Eq. TFW; one amplitude,
p = 1) with the FP64 oracle on the same seeded inputs: the Thomas-Fermi term
of the potential kernel, the von Weizsaecker-weighted stencil, the closed-form
p = 1 Cayley step (Lemma 3.1 (3)), the energy and gradient, and whole
minimisations in FP64 and in mixed precision."""
import math

import numpy as np
import pytest

import ks_inputs as ki
from oracle import energy as oe
from oracle import fe as ofe
from oracle import stiefel as ost

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-12


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def assert_rel(got, want, rel=REL, what=""):
    got, want = np.asarray(got), np.asarray(want)
    err = np.abs(got - want).max() / max(np.abs(want).max(), 1e-300)
    assert err <= rel, f"{what}: max error {err:.3e} relative to max |want| > {rel:.1e}"


# n = 13^3 and 17^3: ragged against the 16 x 64 node tile of the one-amplitude
# stencil in both x and y; mu = 1 with the lumped mass, and a weak von
# Weizsaecker term with the consistent Q1 mass
OF_CASES = [dict(N=13, L=7.0, natoms=2, Z=2.0, seed=11, mu=1.0, mass=1),
            dict(N=17, L=8.0, natoms=3, Z=1.0, seed=12, mu=0.2, mass=0)]


@pytest.fixture(params=OF_CASES, ids=["N13mu1-lumped", "N17mu0.2-consistent"])
def case(request):
    s = ki.small_of_system(**request.param)
    model = oe.Model.from_system(s)
    c = ost.m_orthonormalize(model, s.x0())
    return s, model, c


def make(s, **kw):
    import paper_1308_2864_gb300 as ks
    return ks.Problem.from_system(s, **kw)


def test_of_potential_adds_thomas_fermi(case):
    s, model, c = case
    P = make(s)
    rho = oe.density(c, model.occ)
    vH = ofe.poisson_exact(4 * math.pi * model.h ** 3 * rho, model.N, model.h)
    veff, e = P.step_potential(dev(rho), dev(vH))
    eps, vxc = oe.lda(rho, model.xc)
    etf, vtf = oe.thomas_fermi(rho)
    h3 = model.h ** 3
    assert_rel(host(veff), model.vext() + vH + vxc + vtf, what="veff")
    assert e[2] == pytest.approx(h3 * rho @ eps, rel=REL)
    assert e[3] == pytest.approx(h3 * np.sum(etf), rel=REL)


def test_of_stencil_weights_the_kinetic_term(case):
    s, model, c = case
    P = make(s)
    rng = np.random.default_rng(2)
    veff = rng.standard_normal(model.n)
    EX, MX, kin = P.step_hamiltonian(dev(c), dev(veff))
    Kc = ofe.apply_K(c, model.N, model.h)
    f, mu = model.occ, model.mu
    assert_rel(host(EX), mu * f * Kc + 2 * f * model.h ** 3 * veff[:, None] * c, what="E_c")
    assert_rel(host(MX), model.apply_M(c), what="M c")
    assert kin == pytest.approx(0.5 * mu * f * float(np.sum(c * Kc)), rel=REL)


def test_of_energy_grad(case):
    s, model, c = case
    P = make(s, cg_tol=1e-13)
    E, EX, D, g = P.energy_grad(dev(c), want_ex=True, want_d=True)
    ref = oe.evaluate(model, c)
    pt = ost.project(model, c, ref)
    assert E == pytest.approx(ref.E, rel=1e-12)
    assert_rel(host(EX), ref.EX, rel=1e-11, what="E_c")
    assert_rel(host(D), pt.D, rel=1e-10, what="D")
    assert g == pytest.approx(pt.dnorm, rel=1e-10)
    for got, key in zip(P.energy_parts(), ["kinetic", "external", "hartree", "xc", "ion"]):
        assert got == pytest.approx(ref.parts[key], rel=1e-11, abs=1e-12)


@pytest.mark.parametrize("kind", ["qr", "cayley"])
def test_of_retract(case, kind):
    import paper_1308_2864_gb300 as ks
    s, model, c = case
    P = make(s)
    ref = oe.evaluate(model, c)
    pt = ost.project(model, c, ref)
    for tau in (1e-3, 0.05, 2.0):
        got = host(P.retract(ks.KS_QR if kind == "qr" else ks.KS_CAYLEY, dev(c), dev(ref.EX), tau))
        want = (ost.retract_qr if kind == "qr" else ost.retract_cayley_p1)(model, pt, tau)
        assert_rel(got, want, rel=1e-11, what=f"{kind} tau={tau}")
        assert ost.ortho_error(model, got) < 1e-12


def _converged_case():
    s = ki.small_of_system(N=11, L=7.0, natoms=2, Z=1.0, seed=11, mu=1.0)
    return s, oe.Model.from_system(s)


@pytest.mark.parametrize("retraction", ["qr", "cayley"])
def test_of_minimize_matches_oracle(retraction):
    s, model = _converged_case()
    ref = ost.minimize(model, s.x0(), ost.Options(retraction=retraction, gtol=1e-8, maxit=3000))
    assert ref.converged
    P = make(s)
    c = dev(s.x0())
    r = P.minimize(c, retraction=retraction, gtol=1e-8, maxit=3000)
    assert r["status"] == 0 and r["gradnorm"] <= 1e-8
    assert r["E"] == pytest.approx(ref.E, abs=1e-8)
    cg = host(c)
    assert ost.ortho_error(model, cg) < 1e-12
    # the density is unique (the amplitude only up to sign)
    assert_rel(oe.density(cg, model.occ), oe.density(ref.X, model.occ), rel=1e-6, what="rho")


@pytest.mark.parametrize("retraction", ["qr", "cayley"])
def test_of_mixed_precision_then_polish(retraction):
    s, model = _converged_case()
    ref = ost.minimize(model, s.x0(), ost.Options(retraction=retraction, gtol=1e-8, maxit=3000))
    P = make(s)
    c = dev(s.x0())
    r = P.minimize(c, retraction=retraction, gtol=1e-8, maxit=4000, precision="mixed",
                   polish_gtol=1e-4)
    assert r["status"] == 0 and r["gradnorm"] <= 1e-8
    assert r["mixed_iters"] > 0
    assert r["E"] == pytest.approx(ref.E, abs=1e-8)


@pytest.mark.parametrize("retraction", ["qr", "cayley"])
def test_lumped_mass_kohn_sham(retraction):
    # the lumped metric with orbitals (p = 3): one step's pieces and a whole
    # minimisation against the oracle under the same metric
    import paper_1308_2864_gb300 as ks
    s = ki.small_system(N=10, L=7.0, natoms=2, p=3, Z=1.5, seed=7)
    s.rc, s.mass = 1.0, 1
    model = oe.Model.from_system(s)
    X = ost.m_orthonormalize(model, s.x0())
    P = make(s, cg_tol=1e-13)
    E, EX, D, g = P.energy_grad(dev(X), want_ex=True, want_d=True)
    ref = oe.evaluate(model, X)
    pt = ost.project(model, X, ref)
    assert E == pytest.approx(ref.E, rel=1e-12)
    assert_rel(host(D), pt.D, rel=1e-10, what="D")
    assert_rel(host(P.step_mass_inverse(dev(ref.EX))), pt.G, rel=1e-13, what="M^-1 E_X")
    got = host(P.retract(ks.KS_QR if retraction == "qr" else ks.KS_CAYLEY, dev(X), dev(ref.EX), 0.05))
    want = (ost.retract_qr if retraction == "qr" else ost.retract_cayley)(model, pt, 0.05)
    assert_rel(got, want, rel=1e-11, what="retraction")
    r_ref = ost.minimize(model, s.x0(), ost.Options(retraction=retraction, gtol=1e-8, maxit=3000))
    P2 = make(s)
    Xd = dev(s.x0())
    r = P2.minimize(Xd, retraction=retraction, gtol=1e-8, maxit=3000)
    assert r["status"] == 0 and r_ref.converged
    assert r["E"] == pytest.approx(r_ref.E, abs=1e-8)
    # under the lumped metric the nodal density integrates to the electron count
    rho = oe.density(host(Xd), model.occ)
    assert model.h ** 3 * rho.sum() == pytest.approx(model.occ * s.p, rel=1e-12)


def test_of_descriptions_are_checked():
    import paper_1308_2864_gb300 as ks
    s = ki.small_system(N=6, L=6.0, natoms=1, p=2)
    with pytest.raises(ks.KSError):
        ks.Problem.from_system(s, kinetic=ks.KS_KIN_TFW)        # p must be 1
    of = ki.small_of_system(N=6)
    with pytest.raises(ks.KSError):
        ks.Problem.from_system(of, mu=-1.0)
    with pytest.raises(ks.KSError):
        ks.Batch([of])                                          # single-system path only
