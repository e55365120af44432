"""Pins of the oracle's orbital-free model (Sec. 2.2: Eq. TFW, Eq. OFeng,
Eq. OF_euler; discretised as Eq. disOFinf and minimised as Eq. OFDFT-y on
the unit sphere of the M metric, here the lumped mass h^3 I) against the
free-electron gas, a continuum closed form, finite differences, the V = 0
spectrum and a dense SCF."""
import math

import numpy as np
import pytest

import ks_inputs as ki
from oracle import brute, energy, fe, stiefel


def _of_model(N=6, L=6.0, natoms=2, Z=1.0, seed=11, mu=1.0, **kw):
    s = ki.small_of_system(N=N, L=L, natoms=natoms, Z=Z, seed=seed, mu=mu)
    return energy.Model.from_system(s, **kw), s


def test_thomas_fermi_is_the_free_electron_gas():
    # Free electron gas of density rho: k_F = (3 pi^2 rho)^(1/3), Fermi
    # energy k_F^2 / 2, mean kinetic energy per electron (3/5) of it.
    rho = np.array([1e-4, 0.01, 0.3, 1.0, 7.5])
    kf = (3.0 * math.pi ** 2 * rho) ** (1.0 / 3.0)
    e, _ = energy.thomas_fermi(rho)
    assert np.allclose(e, rho * 0.6 * 0.5 * kf ** 2, rtol=1e-14)
    # the textbook value of the constant, C_F = 2.871 hartree bohr^2
    assert energy.C_TF == pytest.approx(2.8712, abs=5e-5)
    assert energy.thomas_fermi(np.array([0.0, 1e-31]))[0].tolist() == [0.0, 0.0]


def test_thomas_fermi_potential_is_the_derivative():
    rho = np.array([1e-3, 0.05, 0.7, 3.0])
    d = 1e-6 * rho
    fd = (energy.thomas_fermi(rho + d)[0] - energy.thomas_fermi(rho - d)[0]) / (2 * d)
    assert np.allclose(energy.thomas_fermi(rho)[1], fd, rtol=1e-8)


def test_von_weizsaecker_term_converges_to_the_continuum_integral():
    # phi = sqrt(f) prod sin(pi x_i / L) on the cube with zero Dirichlet
    # data: (1/8) int |grad rho|^2 / rho = (f/2) int |grad(phi/sqrt f)|^2
    # = (f/2) 3 (pi/L)^2 (L/2)^3.  The discrete (f/2) c^T K c of the sampled
    # amplitude (the Q1 interpolant's exact integral) converges at second order.
    L, f = 5.0, 3.0
    want = 0.5 * f * 3.0 * (math.pi / L) ** 2 * (L / 2.0) ** 3
    errs = []
    for N in (15, 31):
        h = L / (N + 1)
        g = (np.arange(N) + 1.0) * h
        z, y, x = np.meshgrid(g, g, g, indexing="ij")
        c = (np.sin(math.pi * x / L) * np.sin(math.pi * y / L) * np.sin(math.pi * z / L)).reshape(-1, 1)
        model = energy.Model(N=N, L=L, atoms=np.zeros((0, 3)), Z=np.zeros(0), p=1, occ=f,
                             kinetic=energy.KIN_TFW, mu=1.0, use_tf=False, use_ext=False,
                             use_hartree=False, use_xc=False)
        ev = energy.evaluate(model, c)
        errs.append(abs(ev.parts["kinetic"] - want) / want)
    assert errs[1] < 5e-3
    assert 3.5 < errs[0] / errs[1] < 4.5


@pytest.mark.parametrize("terms", [
    dict(use_ext=False, use_hartree=False, use_xc=False),
    dict(use_hartree=False, use_xc=False),
    dict(use_tf=False),
    dict(mu=0.2),
    dict(),
])
def test_of_gradient_central_difference(terms):
    mu = terms.pop("mu", 1.0)
    model, s = _of_model(mu=mu, **terms)
    rng = np.random.default_rng(12)
    c = s.x0() * 0.2
    dc = rng.standard_normal(c.shape)
    ev = energy.evaluate(model, c)

    def cd(eps):
        return (energy.evaluate(model, c + eps * dc).E
                - energy.evaluate(model, c - eps * dc).E) / (2 * eps)

    # Richardson extrapolation of the central difference (error O(eps^4)):
    # rho^(5/3) = f^(5/3) c^(10/3) has a large third derivative at c ~ 0.2
    eps = 1e-4
    fd = (4.0 * cd(eps / 2) - cd(eps)) / 3.0
    assert float(np.sum(ev.EX * dc)) == pytest.approx(fd, rel=1e-9)


def test_of_parts():
    # a von Weizsaecker weight other than 1, so that the weight is pinned
    model, s = _of_model(mu=0.37)
    c = stiefel.m_orthonormalize(model, s.x0())
    ev = energy.evaluate(model, c)
    assert ev.E == pytest.approx(sum(ev.parts.values()), rel=1e-15)
    # kinetic = mu vW + TF, both positive; the TF part alone from the density
    rho = energy.density(c, model.occ)
    tf = model.h ** 3 * float(np.sum(energy.thomas_fermi(rho)[0]))
    KX = fe.apply_K(c, model.N, model.h)
    vw = 0.5 * model.occ * float(np.sum(c * KX))
    assert model.mu == 0.37
    assert ev.parts["kinetic"] == pytest.approx(0.37 * vw + tf, rel=1e-14)
    assert tf > 0 and vw > 0
    # the electron count the constraint fixes, f c^T M c = N_e, is the
    # integral of the nodal density under the lumped mass
    ne = float(np.sum(model.Z))
    assert model.occ * float(c[:, 0] @ model.apply_M(c)[:, 0]) == pytest.approx(ne, rel=1e-13)
    assert model.h ** 3 * float(np.sum(rho)) == pytest.approx(ne, rel=1e-13)


def test_consistent_mass_lets_the_nodal_density_grow():
    # Why the orbital-free systems take the lumped mass: under the consistent
    # Q1 mass an amplitude oscillating node to node has c^T M c = 1 while its
    # nodal density integrates to (3 / (2 + cos t))^3 -> 27 times the electron
    # count (the M1 eigenvalue (h/3)(2 + cos t) of the highest sine mode against
    # h for the row sums), a gain the external potential can exploit.
    N, L = 9, 5.0
    h = L / (N + 1)
    i = np.arange(N)
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    t = np.pi * N / (N + 1)
    phi = lambda k: np.sin((k + 1) * t)                     # highest 1-D sine mode
    c = (phi(x) * phi(y) * phi(z)).reshape(-1, 1)
    m = energy.Model(N=N, L=L, atoms=np.zeros((0, 3)), Z=np.zeros(0), p=1, occ=1.0)
    c = c / math.sqrt(float(c[:, 0] @ m.apply_M(c)[:, 0]))
    lumped = h ** 3 * float(np.sum(c * c))
    assert lumped == pytest.approx((3.0 / (2.0 + math.cos(t))) ** 3, rel=1e-12)
    assert lumped > 20


def test_tfw_model_needs_one_amplitude():
    s = ki.small_system(N=4, L=4.0, natoms=1, p=2)
    with pytest.raises(ValueError):
        energy.Model.from_system(s, kinetic=energy.KIN_TFW)


@pytest.mark.parametrize("retraction", ["qr", "cayley"])
def test_of_v0_minimiser_is_the_lowest_mode(retraction):
    # vW only, V = 0: min mu (f/2) c^T K c on c^T M c = 1 is mu (f/2) lambda_1,
    # the (1,1,1) generalised eigenvalue of (K, M).
    model, s = _of_model(N=6, mu=0.5, use_tf=False, use_ext=False, use_hartree=False,
                         use_xc=False)
    # lowest eigenvalue of K against h^3 I: K's (1,1,1) sine mode,
    # 3 kappa_1 mu_1^2 (K = K1 M1 M1 + M1 K1 M1 + M1 M1 K1)
    kap, mu1 = fe.eigen_1d(model.N, model.h)
    want = 0.5 * model.mu * model.occ * 3.0 * kap[0] * mu1[0] ** 2 / model.h ** 3
    r = stiefel.minimize(model, s.x0(), stiefel.Options(retraction=retraction, gtol=1e-9,
                                                        maxit=2000))
    assert r.converged
    assert r.E == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("retraction", ["qr", "cayley"])
@pytest.mark.parametrize("Z,natoms", [(1.0, 2), (2.0, 1), (1.5, 2)])
def test_of_minimiser_matches_dense_scf(retraction, Z, natoms):
    # All terms (TF + vW + external + Hartree + Slater/PZ81), mu = 1.  The
    # direct minimiser's amplitude is the lowest mode of the dense Eq. OF_euler
    # operator it generates (H c = lambda_1 M c, one sign), and a damped SCF
    # with linear density mixing reaches the same energy.  (With mu = 0.2 on
    # this 0.86 bohr grid the discrete minima change sign and the SCF does not
    # settle: no nodeless reference exists there.)
    model, s = _of_model(N=6, L=6.0, natoms=natoms, Z=Z, mu=1.0)
    r = stiefel.minimize(model, s.x0(), stiefel.Options(retraction=retraction, gtol=1e-9,
                                                        maxit=4000))
    assert r.converged
    H = brute.hamiltonian_dense(model, energy.density(r.X, model.occ))
    M = model.dense_M()
    w, V = brute.lowest_pencil(H, M, 1)
    lam = float(r.X[:, 0] @ H @ r.X[:, 0])
    assert np.abs(H @ r.X[:, 0] - lam * (M @ r.X[:, 0])).max() < 1e-7
    assert lam == pytest.approx(w[0], abs=1e-8)
    assert abs(abs(float(V[:, 0] @ M @ r.X[:, 0])) - 1.0) < 1e-8
    # the ground-state amplitude has one sign (no node)
    assert np.all(r.X[:, 0] > 0) or np.all(r.X[:, 0] < 0)
    E_scf, _, _ = brute.scf_reference(model)
    assert r.E == pytest.approx(E_scf, abs=1e-10)
