"""Pins of the oracle's uniform refinement (Alg. AdpConOptM with every
element refined, Sec. 4.3): the Q1 prolongation against brute-force
evaluation of the trilinear interpolant, the Galerkin identities of nested
Q1 spaces, and the continuation reaching the single-grid minimiser."""
import math

import numpy as np
import pytest

import ks_inputs as ki
from oracle import energy, fe, stiefel


def _hat(t: np.ndarray, h: float) -> np.ndarray:
    return np.maximum(0.0, 1.0 - np.abs(t) / h)


def test_prolong_is_the_trilinear_interpolant():
    # the coarse field's Q1 interpolant sum_i c_i prod_d hat((x_d - X_i,d)/h_c),
    # evaluated at every fine node by brute force
    L, Nc = 4.0, 3
    Nf = 2 * Nc + 1
    hc, hf = L / (Nc + 1), L / (Nf + 1)
    rng = np.random.default_rng(3)
    c = rng.standard_normal((Nc ** 3, 2))
    gc = (np.arange(Nc) + 1.0) * hc
    gf = (np.arange(Nf) + 1.0) * hf
    want = np.zeros((Nf ** 3, 2))
    for kz in range(Nf):
        for ky in range(Nf):
            for kx in range(Nf):
                wz, wy, wx = _hat(gf[kz] - gc, hc), _hat(gf[ky] - gc, hc), _hat(gf[kx] - gc, hc)
                w = (wz[:, None, None] * wy[None, :, None] * wx[None, None, :]).reshape(-1)
                want[(kz * Nf + ky) * Nf + kx] = w @ c
    assert np.abs(fe.prolong(c, Nc) - want).max() < 1e-14


@pytest.mark.parametrize("Nc", [2, 3])
def test_prolong_galerkin_identities(Nc):
    # nested Q1 spaces: the coarse function and its interpolant are the same
    # function, so P^T K_f P = K_c and P^T M_f P = M_c exactly
    L = 3.0
    Nf = 2 * Nc + 1
    Kc, Mc = fe.dense_K_M(Nc, L / (Nc + 1))
    Kf, Mf = fe.dense_K_M(Nf, L / (Nf + 1))
    P = fe.prolong(np.eye(Nc ** 3), Nc)
    assert np.abs(P.T @ Kf @ P - Kc).max() <= 1e-13 * np.abs(Kc).max()
    assert np.abs(P.T @ Mf @ P - Mc).max() <= 1e-13 * np.abs(Mc).max()


def test_refine_levels():
    assert stiefel.refine_levels(15, 3) == [3, 7, 15]
    assert stiefel.refine_levels(11, 1) == [11]
    with pytest.raises(ValueError):
        stiefel.refine_levels(14, 2)
    with pytest.raises(ValueError):
        stiefel.refine_levels(7, 3)          # coarsest grid would be 1


@pytest.mark.parametrize("kind", ["ks", "of"])
def test_continuation_reaches_the_single_grid_minimiser(kind):
    if kind == "ks":
        s = ki.small_system(N=11, L=7.0, natoms=2, p=2, Z=1.0, seed=7)
        s.rc = 1.0
    else:
        s = ki.small_of_system(N=11, L=7.0, natoms=2, Z=1.0, seed=11)
    model = energy.Model.from_system(s)
    opt = stiefel.Options(retraction="qr", gtol=1e-8, maxit=3000)
    direct = stiefel.minimize(model, s.x0(), opt)
    nc = 5 ** 3                              # the coarse grid of refine_levels(11, 2)
    x0 = (ki.initial_orbitals(s.seed, 0, nc, s.p) if kind == "ks"
          else ki.initial_density_amplitude(s.seed, 0, nc))
    res = stiefel.minimize_refine(model, x0, 2, opt, coarse_gtol=1e-3)
    assert [r.X.shape[0] for r in res] == [5 ** 3, 11 ** 3]
    assert res[0].dnorm <= 1e-3 and res[1].converged
    assert res[1].E == pytest.approx(direct.E, abs=1e-8)
    assert stiefel.ortho_error(model, res[1].X) < 1e-12
