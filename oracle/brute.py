"""Dense brute-force references on tiny grids, used only to pin the oracle.

  * lowest generalised eigenpairs of a dense symmetric pencil (H, M);
  * the SCF fixed point of Alg. SCF (Sec. 2.4) with plain linear density
    mixing and dense eigensolves, converged far below the tolerance of the
    direct minimiser.  At an SCF fixed point with the p lowest states
    occupied, H(X) X = M X Lambda holds (Eq. disKS with the mass metric), so
    the direct minimiser must reach the same energy.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import eigh

from . import fe
from .energy import KIN_TFW, Model, lda, density, evaluate, thomas_fermi


def lowest_pencil(H: np.ndarray, M: np.ndarray, p: int):
    w, V = eigh(H, M, subset_by_index=[0, p - 1])
    return w, V


def hamiltonian_dense(model: Model, rho: np.ndarray) -> np.ndarray:
    """H(rho) = K/2 + h^3 Diag(Vext + vH(rho) + v_xc(rho)); E_X = 2 f H X.
    Orbital-free (TFW): H = mu K/2 + h^3 Diag(Vext + vH + v_xc + v_TF), the
    discrete operator of Eq. OF_euler."""
    K, _ = fe.dense_K_M(model.N, model.h)
    h3 = model.h ** 3
    veff = model.vext().copy()
    if model.kinetic == KIN_TFW and model.use_tf:
        veff += thomas_fermi(rho)[1]
    if model.use_hartree:
        veff += fe.poisson_exact(4.0 * np.pi * h3 * rho, model.N, model.h)
    if model.use_xc:
        veff += lda(rho, model.xc)[1]
    return 0.5 * model.kin_weight * K + h3 * np.diag(veff)


def scf_reference(model: Model, alpha: float = 0.3, tol: float = 1e-13,
                  maxit: int = 5000):
    """Damped SCF: rho_in -> lowest p eigenvectors of (H(rho_in), M) ->
    rho_out; rho_in <- (1-alpha) rho_in + alpha rho_out until
    max|rho_out - rho_in| <= tol.  Returns (E, X, eigenvalues)."""
    M = model.dense_M()
    m0 = Model(**{**model.__dict__, "use_hartree": False, "use_xc": False})
    w, X = lowest_pencil(hamiltonian_dense(m0, np.zeros(model.n)), M, model.p)
    rho_in = density(X, model.occ)
    for _ in range(maxit):
        w, X = lowest_pencil(hamiltonian_dense(model, rho_in), M, model.p)
        rho_out = density(X, model.occ)
        if np.max(np.abs(rho_out - rho_in)) <= tol:
            break
        rho_in = (1.0 - alpha) * rho_in + alpha * rho_out
    else:
        raise RuntimeError("SCF reference did not converge")
    return evaluate(model, X).E, X, w
