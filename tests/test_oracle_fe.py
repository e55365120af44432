"""Pins of the oracle's Q1 discretisation (Sec. 2.3 restated for Q1 finite
elements) against closed forms and independent formulations."""
import math

import numpy as np
import pytest

from oracle import fe


def test_stencil_textbook_coefficients():
    # Trilinear (Q1) Laplacian on a uniform grid: (h/12) * [32 centre, 0 face,
    # -2 edge, -1 corner]; mass: (h^3/216) * [64, 16, 4, 1].
    h = 0.37
    kc, mc = fe.stencil_coefficients(h)
    for off, c in kc.items():
        nz = sum(1 for d in off if d != 0)
        want = {0: 32.0, 1: 0.0, 2: -2.0, 3: -1.0}[nz] * h / 12.0
        assert c == pytest.approx(want, abs=1e-15)
        assert mc[off] == pytest.approx({0: 64, 1: 16, 2: 4, 3: 1}[nz] * h ** 3 / 216.0, rel=1e-14)


@pytest.mark.parametrize("N", [3, 5])
def test_stencil_matches_kronecker(N):
    h = 1.0 / (N + 1)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((N ** 3, 3))
    K, M = fe.dense_K_M(N, h)
    assert np.abs(fe.apply_K(X, N, h) - K @ X).max() < 1e-13
    assert np.abs(fe.apply_M(X, N, h) - M @ X).max() < 1e-15


def test_row_sums_interior():
    N, h = 7, 0.3
    K, M = fe.dense_K_M(N, h)
    k = (3 * N + 3) * N + 3          # centre node: full 27-point row
    assert abs(K[k].sum()) < 1e-14
    assert M[k].sum() == pytest.approx(h ** 3, rel=1e-13)


@pytest.mark.parametrize("N,h", [(4, 0.4), (6, 0.25)])
def test_generalized_eigenvalues_closed_form(N, h):
    from scipy.linalg import eigh
    K, M = fe.dense_K_M(N, h)
    w = eigh(K, M, eigvals_only=True)
    assert np.allclose(w, fe.generalized_eigs_closed_form(N, h), rtol=1e-11, atol=1e-11)


def test_sine_basis_diagonalises_1d():
    N, h = 9, 0.2
    Phi = fe.sine_basis(N)
    K1, M1 = fe.q1_1d(N, h)
    kap, mu = fe.eigen_1d(N, h)
    assert np.allclose(Phi @ Phi, np.eye(N), atol=1e-14)
    assert np.allclose(Phi @ K1 @ Phi, np.diag(kap), atol=1e-12)
    assert np.allclose(Phi @ M1 @ Phi, np.diag(mu), atol=1e-14)


def test_mass_inverse_two_ways():
    N, h = 8, 0.3
    rng = np.random.default_rng(5)
    E = rng.standard_normal((N ** 3, 4))
    G = fe.mass_inverse(E, N, h)
    assert np.abs(fe.apply_M(G, N, h) - E).max() < 1e-12 * np.abs(E).max()
    assert np.allclose(G, fe.mass_inverse_sine(E, N, h), rtol=1e-11, atol=1e-11)


def test_poisson_exact_and_cg():
    N, h = 9, 0.25
    rng = np.random.default_rng(8)
    b = rng.random(N ** 3)
    v = fe.poisson_exact(b, N, h)
    assert np.abs(fe.apply_K(v, N, h) - b).max() < 1e-12
    K, _ = fe.dense_K_M(N, h)
    assert np.allclose(v, np.linalg.solve(K, b), rtol=1e-10)
    vc, r, it, ok = fe.cg_solve(lambda x: fe.apply_K(x, N, h), b, None, 1e-12, 1000)
    assert ok and it > 5
    assert np.allclose(vc, v, rtol=1e-9, atol=1e-11)
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(b) * 1.0001


def _continuum_hartree_gaussian(L, x0, sigma, q, nmodes=80):
    """Exact E_H = 1/2 int rho v of a separable Gaussian charge in a grounded
    cube (-Lap v = 4 pi rho, v = 0 on the faces) by its sine series."""
    a = np.arange(1, nmodes + 1)
    ghat = [(2.0 / L) * np.exp(-0.5 * (a * np.pi * sigma / L) ** 2) * np.sin(a * np.pi * c / L)
            for c in x0]
    k2 = (np.pi / L) ** 2 * (a[:, None, None] ** 2 + a[None, :, None] ** 2 + a[None, None, :] ** 2)
    rhat = q * ghat[0][:, None, None] * ghat[1][None, :, None] * ghat[2][None, None, :]
    return 0.5 * (L / 2.0) ** 3 * float(np.sum(4.0 * np.pi * rhat ** 2 / k2))


def test_hartree_energy_converges_to_continuum():
    # The discrete Hartree term 1/2 h^3 rho^T vH with K vH = 4 pi h^3 rho must
    # converge (O(h^2)) to the continuum Coulomb energy of the same charge.
    from oracle.energy import node_coords
    L, sigma, q = 8.0, 0.7, 1.0
    x0 = (3.9, 4.2, 4.05)
    exact = _continuum_hartree_gaussian(L, x0, sigma, q)
    errs = []
    for N in (15, 31):
        h = L / (N + 1)
        r = node_coords(N, h)
        d2 = np.sum((r - np.array(x0)) ** 2, axis=1)
        rho = q * np.exp(-0.5 * d2 / sigma ** 2) / (sigma * math.sqrt(2 * math.pi)) ** 3
        v = fe.poisson_exact(4 * math.pi * h ** 3 * rho, N, h)
        errs.append(abs(0.5 * h ** 3 * (rho @ v) - exact) / exact)
    # second-order convergence: halving h divides the error by about 4
    assert errs[1] < 0.02
    assert 3.5 < errs[0] / errs[1] < 4.6
