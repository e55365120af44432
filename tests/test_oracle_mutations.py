"""The oracle's pins catch plausible mistakes.  Each case plants one mistake
in the oracle (on the CPU, through monkeypatch): a dropped term or factor, a
flipped sign, a transposed operand, a wrong boundary.  It then checks that
at least one of the pins named for it fails, and that the same pins pass
without the mistake."""
import numpy as np
import pytest

from oracle import energy, fe, stiefel

import test_oracle_energy as pen
import test_oracle_fe as pfe
import test_oracle_ofdft as pof
import test_oracle_refine as pre
import test_oracle_stiefel as pst

CAUGHT = (AssertionError, RuntimeError, np.linalg.LinAlgError)


def first_failure(pins):
    """Index of the first pin that fails, or None when all pass."""
    for i, pin in enumerate(pins):
        try:
            pin()
        except CAUGHT:
            return i
    return None


# ---------------------------------------------------------------- mistakes

def m1_offdiag_quarter(mp):
    mp.setattr(fe, "m1_entry", lambda d, h: 4.0 * h / 6.0 if d == 0 else h / 4.0)


def k1_offdiag_sign(mp):
    mp.setattr(fe, "k1_entry", lambda d, h: 2.0 / h if d == 0 else 1.0 / h)


def k_without_z_term(mp):
    def coef(h):
        kc, mc = {}, {}
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    kc[(dz, dy, dx)] = (fe.k1_entry(dx, h) * fe.m1_entry(dy, h) * fe.m1_entry(dz, h)
                                        + fe.m1_entry(dx, h) * fe.k1_entry(dy, h) * fe.m1_entry(dz, h))
                    mc[(dz, dy, dx)] = fe.m1_entry(dx, h) * fe.m1_entry(dy, h) * fe.m1_entry(dz, h)
        return kc, mc
    mp.setattr(fe, "stencil_coefficients", coef)


def periodic_boundary(mp):
    def apply(X, N, coef):
        X = np.asarray(X, dtype=np.float64)
        squeeze = X.ndim == 1
        X2 = X[:, None] if squeeze else X
        p = X2.shape[1]
        G = X2.reshape(N, N, N, p)
        out = np.zeros_like(G)
        for (dz, dy, dx), c in coef.items():
            out += c * np.roll(G, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
        out = out.reshape(N ** 3, p)
        return out[:, 0] if squeeze else out
    mp.setattr(fe, "apply_stencil", apply)


def density_without_occupation(mp):
    mp.setattr(energy, "density", lambda X, occ: np.einsum("ki,ki->k", X, X))


def slater_potential_is_energy_density(mp):
    orig = energy.slater
    mp.setattr(energy, "slater", lambda rho: (orig(rho)[0], orig(rho)[0]))


def pz81_beta2_sign(mp):
    mp.setattr(energy, "PZ_BETA2", -energy.PZ_BETA2)


def pz81_beta2_digits_transposed(mp):
    mp.setattr(energy, "PZ_BETA2", 0.3343)


def eii_double_counted(mp):
    orig = energy.e_ii
    mp.setattr(energy, "e_ii", lambda atoms, Z: 2.0 * orig(atoms, Z))


def hartree_without_4pi(mp):
    def hartree(model, rho, v_guess=None):
        v = fe.poisson_exact(model.h ** 3 * rho, model.N, model.h)
        return v, np.zeros_like(rho), 0
    mp.setattr(energy, "hartree", hartree)


def vext_sign(mp):
    orig = energy.v_ext
    mp.setattr(energy, "v_ext", lambda *a: -orig(*a))


def gradient_potential_without_factor_2(mp):
    orig = energy.evaluate

    def evaluate(model, X, v_guess=None):
        ev = orig(model, X, v_guess)
        ev.EX = ev.EX - model.occ * model.h ** 3 * ev.veff[:, None] * np.asarray(X)
        return ev
    mp.setattr(energy, "evaluate", evaluate)
    mp.setattr(stiefel, "evaluate", evaluate)


def projection_without_the_metric(mp):
    # D = E_X - X S (the plain Stiefel form, M = I) instead of M^-1 E_X - X S.
    # (Transposing S is no mistake here: E_X = H(X) X with H symmetric makes
    # X^T E_X symmetric on every X.)
    orig = stiefel.project

    def project(model, X, ev):
        pt = orig(model, X, ev)
        D = ev.EX - X @ pt.S
        MD = model.apply_M(D)
        return stiefel.Point(X=X, MX=pt.MX, ev=ev, G=pt.G, S=pt.S, D=D, MD=MD,
                             dnorm2=float(np.sum(D * MD)))
    mp.setattr(stiefel, "project", project)


def qr_moves_uphill(mp):
    from scipy.linalg import cholesky, solve_triangular

    def retract(model, pt, tau):
        Y = pt.X + tau * pt.D
        R = Y.T @ model.apply_M(Y)
        Lc = cholesky(0.5 * (R + R.T), lower=True)
        return solve_triangular(Lc, Y.T, lower=True).T
    mp.setattr(stiefel, "retract_qr", retract)


def cayley_inverse_sign(mp):
    from scipy.linalg import solve

    def retract(model, pt, tau):
        U, VU, VY = stiefel.cayley_blocks(model, pt)
        P = solve(np.eye(VU.shape[0]) - 0.5 * tau * VU, VY)
        return pt.X - tau * (U @ P)
    mp.setattr(stiefel, "retract_cayley", retract)


def cayley_p1_dropped_term(mp):
    # beta2 without its second-order part tau/2 (ax^2 - aa xx)
    def retract(model, pt, tau):
        x, g = pt.X[:, 0], pt.G[:, 0]
        ax = float(pt.ev.EX[:, 0] @ x)
        aa = float(pt.ev.EX[:, 0] @ g)
        xx = float(x @ pt.MX[:, 0])
        t2 = (0.5 * tau) ** 2
        den = 1.0 - t2 * ax * ax + t2 * aa * xx
        beta1 = tau * xx / den
        beta2 = -tau * ax / den
        return (x - beta1 * g - beta2 * x)[:, None]
    mp.setattr(stiefel, "retract_cayley_p1", retract)


def bb_rules_swapped(mp):
    orig = stiefel.bb_step
    mp.setattr(stiefel, "bb_step", lambda k, ss, sy, yy, opt: orig(k + 1, ss, sy, yy, opt))


def mass_inverse_is_mass(mp):
    mp.setattr(fe, "mass_inverse", lambda E, N, h: fe.apply_M(E, N, h))


def poisson_missing_a_power_of_h(mp):
    orig = fe.poisson_exact
    mp.setattr(fe, "poisson_exact", lambda b, N, h: h * orig(b, N, h))


def thomas_fermi_constant_doubled(mp):
    mp.setattr(energy, "C_TF", 2.0 * energy.C_TF)


def prolong_midpoints_quartered(mp):
    orig = fe.prolong_1d

    def p1(Nc):
        P = orig(Nc)
        P[P == 0.5] = 0.25
        return P
    mp.setattr(fe, "prolong_1d", p1)


def vw_weight_ignored(mp):
    mp.setattr(energy.Model, "kin_weight", property(lambda self: 1.0))


def lumped_mass_ignored(mp):
    mp.setattr(energy.Model, "apply_M", lambda self, X: fe.apply_M(X, self.N, self.h))


def tf_potential_without_five_thirds(mp):
    orig = energy.thomas_fermi
    mp.setattr(energy, "thomas_fermi", lambda rho: (orig(rho)[0], 0.6 * orig(rho)[1]))


SCF_CASE = dict(N=7, L=6.0, natoms=1, p=1, Z=2.0, seed=7)
EXT_ONLY = dict(use_hartree=False, use_xc=False)

CASES = {
    "mass off-diagonal h/4": (m1_offdiag_quarter, [pfe.test_stencil_textbook_coefficients]),
    "stiffness off-diagonal sign": (k1_offdiag_sign, [pfe.test_stencil_textbook_coefficients,
                                                      pfe.test_row_sums_interior]),
    "stiffness without its z term": (k_without_z_term,
                                     [lambda: pfe.test_stencil_matches_kronecker(3)]),
    "periodic instead of Dirichlet": (periodic_boundary,
                                      [lambda: pfe.test_stencil_matches_kronecker(3)]),
    "density without occupation": (density_without_occupation,
                                   [lambda: pen.test_gradient_central_difference(EXT_ONLY)]),
    "v_x equal to eps_x": (slater_potential_is_energy_density,
                           [lambda: pen.test_vxc_is_derivative_of_rho_eps(energy.XC_SLATER)]),
    "PZ81 beta2 sign": (pz81_beta2_sign, [pen.test_pz81_branches_meet_at_rs1]),
    "PZ81 beta2 digits transposed": (
        pz81_beta2_digits_transposed,
        [pen.test_pz81_constants_are_the_published_ones,
         pen.test_pz81_low_density_branch_uses_the_published_parameters]),
    "E_II double counted": (eii_double_counted, [pen.test_eii_two_atoms]),
    "Hartree without 4 pi": (hartree_without_4pi,
                             [lambda: pst.test_minimize_interacting_matches_scf(SCF_CASE, "qr")]),
    "V_ext sign": (vext_sign, [pen.test_vext_coulomb_tail_and_centre]),
    "gradient's potential term without 2": (
        gradient_potential_without_factor_2,
        [lambda: pen.test_gradient_central_difference(EXT_ONLY)]),
    "projection without the metric": (projection_without_the_metric,
                                     [pst.test_gradient_is_tangent_and_matches_y_coordinates]),
    "QR retraction along +D": (
        qr_moves_uphill,
        [lambda: pst.test_retraction_derivative_is_minus_gradient(stiefel.retract_qr)]),
    "Cayley inverse sign": (cayley_inverse_sign,
                            [pst.test_cayley_woodbury_equals_dense_and_preserves_metric]),
    "p = 1 Cayley beta2 term dropped": (cayley_p1_dropped_term, [pst.test_cayley_p1_closed_form]),
    "BB1 and BB2 swapped": (bb_rules_swapped, [pst.test_bb_step_rules]),
    "M^-1 replaced by M": (mass_inverse_is_mass, [pfe.test_mass_inverse_two_ways]),
    "Poisson off by a power of h": (poisson_missing_a_power_of_h,
                                    [pfe.test_poisson_exact_and_cg]),
    "Thomas-Fermi constant doubled": (thomas_fermi_constant_doubled,
                                      [pof.test_thomas_fermi_is_the_free_electron_gas]),
    "prolongation midpoints 1/4": (prolong_midpoints_quartered,
                                   [pre.test_prolong_is_the_trilinear_interpolant]),
    "von Weizsaecker weight ignored": (vw_weight_ignored, [pof.test_of_parts]),
    "lumped mass ignored": (lumped_mass_ignored, [pof.test_of_parts]),
    "v_TF without 5/3": (tf_potential_without_five_thirds,
                         [pof.test_thomas_fermi_potential_is_the_derivative]),
}


@pytest.mark.parametrize("name", list(CASES))
def test_pins_catch_the_planted_mistake(name, monkeypatch):
    plant, pins = CASES[name]
    assert first_failure(pins) is None, "the pins must pass on the intact oracle"
    with monkeypatch.context() as mp:
        plant(mp)
        assert first_failure(pins) is not None, f"no pin caught: {name}"
    assert first_failure(pins) is None
