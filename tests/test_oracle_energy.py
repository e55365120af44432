"""Pins of the oracle's KS functional (Eq. EKS discretised, Sec. 2.3) and its
derivative E_X (Eq. "partial deriv"), LDA, external potential and E_II."""
import math
from pathlib import Path

import numpy as np
import pytest

import ks_inputs as ki
from oracle import energy, fe


def test_slater_uniform_gas_textbook():
    # Uniform electron gas exchange: eps_x = -0.458165.../rs hartree.
    for rs in (0.5, 1.0, 2.0, 5.0):
        rho = 3.0 / (4.0 * math.pi * rs ** 3)
        eps, _ = energy.slater(np.array([rho]))
        assert eps[0] * rs == pytest.approx(-0.4581652932831429, rel=1e-12)


def test_pz81_branches_meet_at_rs1():
    # The two PZ81 branches join at rs = 1 with continuous eps_c and v_c
    # (about -0.0596 and -0.0668 Ha), and the continuity coefficients C, D
    # round to the published 0.0020 and -0.0116.
    rho1 = 3.0 / (4.0 * math.pi)
    below = energy.pz81(np.array([rho1 * (1 + 1e-13)]))
    above = energy.pz81(np.array([rho1 * (1 - 1e-13)]))
    assert below[0][0] == pytest.approx(-0.0596, abs=1e-4)
    assert below[1][0] == pytest.approx(-0.0668, abs=1e-4)
    assert abs(below[0][0] - above[0][0]) < 1e-13
    assert abs(below[1][0] - above[1][0]) < 1e-12
    assert round(energy.PZ_C, 4) == 0.0020 and round(energy.PZ_D, 4) == -0.0116


GOLDEN = Path(__file__).parent / "golden"


def published_pz81():
    """The unpolarised PZ81 parameters as printed in the publication
    (tests/golden/pz81_unpolarized.txt, with its citation)."""
    out = {}
    for line in (GOLDEN / "pz81_unpolarized.txt").read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            name, value = line.split()
            out[name] = float(value)
    return out


def test_pz81_constants_are_the_published_ones():
    # gamma, beta1, beta2, A and B are taken as printed; C and D are the
    # continuity coefficients, which must round to the printed 4 decimals.
    pub = published_pz81()
    assert energy.PZ_GAMMA == pub["gamma"]
    assert energy.PZ_BETA1 == pub["beta1"]
    assert energy.PZ_BETA2 == pub["beta2"]
    assert energy.PZ_A == pub["A"]
    assert energy.PZ_B == pub["B"]
    assert abs(energy.PZ_C - pub["C"]) <= 0.5e-4
    assert abs(energy.PZ_D - pub["D"]) <= 0.5e-4


def test_pz81_low_density_branch_uses_the_published_parameters():
    # On the r_s >= 1 branch eps_c depends only on gamma, beta1 and beta2:
    # evaluated with the printed values it must match the oracle to rounding
    # (a transposed digit in beta2, 0.3334 -> 0.3343, moves eps_c(r_s = 10)
    # by 3e-5 relative).
    pub = published_pz81()
    rs = np.array([1.0, 2.0, 5.0, 10.0, 40.0])
    rho = 3.0 / (4.0 * math.pi * rs ** 3)
    want = pub["gamma"] / (1.0 + pub["beta1"] * np.sqrt(rs) + pub["beta2"] * rs)
    got = energy.pz81(rho * (1.0 - 1e-15))[0]
    np.testing.assert_allclose(got, want, rtol=1e-12)
    # and the r_s < 1 branch at r_s -> 0 follows A ln r_s + B to O(r_s ln r_s)
    r = np.array([1e-6, 1e-7])
    e = energy.pz81(3.0 / (4.0 * math.pi * r ** 3))[0]
    np.testing.assert_allclose(e, pub["A"] * np.log(r) + pub["B"], rtol=0, atol=1e-7)


def test_pz81_energy_is_smooth_across_rs1():
    # one node's density swept through rs = 1: the discrete xc energy has no
    # jump (the rounded published C, D would give 3.2e-5 Ha per electron)
    rho1 = 3.0 / (4.0 * math.pi)
    r = rho1 * (1.0 + np.linspace(-1e-6, 1e-6, 201))
    e = r * energy.lda(r, energy.XC_SLATER_PZ81)[0]
    d = np.diff(e)
    assert np.abs(np.diff(d)).max() < 1e-12


def test_pz81_high_density_limit():
    # Gell-Mann-Brueckner: eps_c -> ((1 - ln 2)/pi^2) ln rs + const as rs -> 0.
    assert energy.PZ_A == pytest.approx((1.0 - math.log(2.0)) / math.pi ** 2, abs=2e-5)
    r1, r2 = 1e-3, 1e-4
    e = energy.pz81(3.0 / (4.0 * math.pi * np.array([r1, r2]) ** 3))[0]
    slope = (e[0] - e[1]) / math.log(r1 / r2)
    assert slope == pytest.approx((1.0 - math.log(2.0)) / math.pi ** 2, rel=5e-3)


@pytest.mark.parametrize("xc", [energy.XC_SLATER, energy.XC_SLATER_PZ81])
def test_vxc_is_derivative_of_rho_eps(xc):
    rho = np.geomspace(1e-5, 50.0, 41)
    eps, v = energy.lda(rho, xc)
    d = 1e-6 * rho
    fp = (rho + d) * energy.lda(rho + d, xc)[0]
    fm = (rho - d) * energy.lda(rho - d, xc)[0]
    fd = (fp - fm) / (2 * d)
    # away from the rs = 1 kink, central differences match to ~1e-8
    rs = np.cbrt(3.0 / (4.0 * math.pi * rho))
    ok = np.abs(rs - 1.0) > 1e-3
    assert np.allclose(v[ok], fd[ok], rtol=1e-7, atol=1e-10)


def test_lda_zero_below_floor():
    eps, v = energy.lda(np.array([0.0, 1e-31]), energy.XC_SLATER_PZ81)
    assert np.all(eps == 0.0) and np.all(v == 0.0)


def test_eii_two_atoms():
    atoms = np.array([[0.0, 0.0, 0.0], [1.5, 2.0, 0.0]])
    assert energy.e_ii(atoms, np.array([4.0, 4.0])) == pytest.approx(16.0 / 2.5, rel=1e-15)
    atoms3 = np.array([[0.0, 0, 0], [3.0, 0, 0], [0, 4.0, 0]])
    want = 1 * 2 / 3.0 + 1 * 3 / 4.0 + 2 * 3 / 5.0
    assert energy.e_ii(atoms3, np.array([1.0, 2.0, 3.0])) == pytest.approx(want, rel=1e-15)


def test_vext_coulomb_tail_and_centre():
    N, h = 9, 0.5
    R = np.array([[2.5, 2.5, 2.5]])          # on node (4, 4, 4)
    V = energy.v_ext(N, h, R, np.array([4.0]), 0.5)
    r = np.linalg.norm(energy.node_coords(N, h) - R, axis=1)
    far = r > 3.5
    assert np.allclose(V[far], -4.0 / r[far], rtol=1e-14)
    k0 = (4 * N + 4) * N + 4
    assert V[k0] == pytest.approx(-4.0 * 2.0 / (math.sqrt(math.pi) * 0.5), rel=1e-14)
    # continuity of the small-r series against erf at r = 1e-6
    from scipy.special import erf
    assert (erf(1e-6 / 0.5) / 1e-6) == pytest.approx(2 / (math.sqrt(math.pi) * 0.5), rel=1e-11)


def _tiny_model(**kw):
    s = ki.small_system(N=6, L=6.0, natoms=2, p=3, Z=2.0, seed=5)
    s.rc = 1.0
    return energy.Model.from_system(s, **kw), s


@pytest.mark.parametrize("terms", [
    dict(use_ext=False, use_hartree=False, use_xc=False),
    dict(use_hartree=False, use_xc=False),
    dict(use_xc=False),
    dict(use_hartree=False),
    dict(),
])
def test_gradient_central_difference(terms):
    model, s = _tiny_model(**terms)
    rng = np.random.default_rng(11)
    X = s.x0() * 0.3
    dX = rng.standard_normal(X.shape)
    ev = energy.evaluate(model, X)
    eps = 1e-5
    fd = (energy.evaluate(model, X + eps * dX).E - energy.evaluate(model, X - eps * dX).E) / (2 * eps)
    an = float(np.sum(ev.EX * dX))
    assert an == pytest.approx(fd, rel=1e-8)


def test_energy_parts_sum_and_signs():
    model, s = _tiny_model()
    ev = energy.evaluate(model, s.x0() * 0.3)
    assert ev.E == pytest.approx(sum(ev.parts.values()), rel=1e-15)
    assert ev.parts["kinetic"] > 0 and ev.parts["hartree"] > 0
    assert ev.parts["external"] < 0 and ev.parts["xc"] < 0 and ev.parts["ion"] > 0


def test_hartree_variational_form_second_order():
    # With an inexact solve the variational Hartree energy errs only to second
    # order in the potential error, the plain 1/2 h^3 rho^T vH to first order.
    model, s = _tiny_model()
    X = s.x0() * 0.3
    rho = energy.density(X, model.occ)
    h3 = model.h ** 3
    b = 4 * math.pi * h3 * rho
    v = fe.poisson_exact(b, model.N, model.h)
    exact = 0.5 * h3 * rho @ v
    rng = np.random.default_rng(2)
    pert = rng.standard_normal(v.shape)
    err_var, err_plain = [], []
    for t in (1e-3, 1e-4):
        vt = v + t * pert
        r = b - fe.apply_K(vt, model.N, model.h)
        err_var.append(abs(0.5 * h3 * rho @ vt + vt @ r / (8 * math.pi) - exact))
        err_plain.append(abs(0.5 * h3 * rho @ vt - exact))
    assert err_var[0] / err_var[1] == pytest.approx(100.0, rel=0.05)
    assert err_plain[0] / err_plain[1] == pytest.approx(10.0, rel=0.05)
