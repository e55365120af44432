"""Q1 finite elements on a uniform cube with homogeneous Dirichlet boundary.

The paper's discrete model (Sec. 2.3) uses a discrete Laplacian L and, for the
finite-element form, a mass matrix B with the constraint c^T B c = 1
(Eq. disOFinf).  Here both are the consistent trilinear (Q1) operators on N
interior nodes per edge, spacing h = L/(N+1):

  1-D:  K1 = (1/h) tridiag(-1, 2, -1),   M1 = (h/6) tridiag(1, 4, 1)
  3-D:  K = K1(x)M1(x)M1 + M1(x)K1(x)M1 + M1(x)M1(x)K1,  M = M1(x)M1(x)M1

The operators are applied here as explicit 27-coefficient sums over the node
neighbourhood (each coefficient is the product of 1-D entries), which is the
plain definition of the assembled stiffness/mass matrices.  The Kronecker
form and the sine eigenbasis below are independent formulations used only
for cross-checks and for exact solves.

Arrays of nodal values are (n, p) with n = N^3, flat node index
k = (iz*N + iy)*N + ix, i.e. reshaped as [iz, iy, ix, orbital].
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_banded


def k1_entry(d: int, h: float) -> float:
    """1-D Q1 stiffness entry at offset d in {-1, 0, 1}."""
    return 2.0 / h if d == 0 else -1.0 / h


def m1_entry(d: int, h: float) -> float:
    """1-D Q1 consistent mass entry at offset d in {-1, 0, 1}."""
    return 4.0 * h / 6.0 if d == 0 else h / 6.0


def stencil_coefficients(h: float) -> tuple[dict, dict]:
    """The 27 coefficients of the 3-D stiffness K and mass M, keyed by the
    offset (dz, dy, dx)."""
    kc, mc = {}, {}
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                kc[(dz, dy, dx)] = (k1_entry(dx, h) * m1_entry(dy, h) * m1_entry(dz, h)
                                    + m1_entry(dx, h) * k1_entry(dy, h) * m1_entry(dz, h)
                                    + m1_entry(dx, h) * m1_entry(dy, h) * k1_entry(dz, h))
                mc[(dz, dy, dx)] = m1_entry(dx, h) * m1_entry(dy, h) * m1_entry(dz, h)
    return kc, mc


def apply_stencil(X: np.ndarray, N: int, coef: dict) -> np.ndarray:
    """out_k = sum over the 27 neighbours k' of k of coef(k'-k) * X_k',
    with X = 0 outside the interior (Dirichlet)."""
    X = np.asarray(X, dtype=np.float64)
    squeeze = X.ndim == 1
    if squeeze:
        X = X[:, None]
    p = X.shape[1]
    pad = np.zeros((N + 2, N + 2, N + 2, p))
    pad[1:-1, 1:-1, 1:-1] = X.reshape(N, N, N, p)
    out = np.zeros((N, N, N, p))
    for (dz, dy, dx), c in coef.items():
        if c == 0.0:
            continue
        out += c * pad[1 + dz:N + 1 + dz, 1 + dy:N + 1 + dy, 1 + dx:N + 1 + dx]
    out = out.reshape(N ** 3, p)
    return out[:, 0] if squeeze else out


def apply_K(X: np.ndarray, N: int, h: float) -> np.ndarray:
    return apply_stencil(X, N, stencil_coefficients(h)[0])


def apply_M(X: np.ndarray, N: int, h: float) -> np.ndarray:
    return apply_stencil(X, N, stencil_coefficients(h)[1])


def q1_1d(N: int, h: float) -> tuple[np.ndarray, np.ndarray]:
    """Dense 1-D K1 and M1 (N x N)."""
    K1 = (2.0 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)) / h
    M1 = (4.0 * np.eye(N) + np.eye(N, k=1) + np.eye(N, k=-1)) * (h / 6.0)
    return K1, M1


def dense_K_M(N: int, h: float) -> tuple[np.ndarray, np.ndarray]:
    """Dense 3-D K and M by Kronecker products (cross-check only; the node
    index has z slowest, so the leftmost factor acts on z)."""
    K1, M1 = q1_1d(N, h)
    K = np.kron(K1, np.kron(M1, M1)) + np.kron(M1, np.kron(K1, M1)) + np.kron(M1, np.kron(M1, K1))
    M = np.kron(M1, np.kron(M1, M1))
    return K, M


def sine_basis(N: int) -> np.ndarray:
    """Orthonormal sine basis Phi_{jk} = sqrt(2/(N+1)) sin(j k pi/(N+1)),
    j, k = 1..N; it diagonalises K1 and M1."""
    j = np.arange(1, N + 1)
    return np.sqrt(2.0 / (N + 1)) * np.sin(np.outer(j, j) * np.pi / (N + 1))


def eigen_1d(N: int, h: float) -> tuple[np.ndarray, np.ndarray]:
    """Eigenvalues of K1 and M1 on the sine basis: kappa_j = (2/h)(1-cos t_j),
    mu_j = (h/3)(2+cos t_j), t_j = j pi/(N+1)."""
    t = np.arange(1, N + 1) * np.pi / (N + 1)
    return (2.0 / h) * (1.0 - np.cos(t)), (h / 3.0) * (2.0 + np.cos(t))


def _along_axes(F: np.ndarray, N: int, A: np.ndarray) -> np.ndarray:
    """Apply the N x N matrix A along each of the three grid axes of F."""
    p = F.shape[1]
    G = F.reshape(N, N, N, p)
    G = np.einsum("az,zyxp->ayxp", A, G)
    G = np.einsum("by,zyxp->zbxp", A, G)
    G = np.einsum("cx,zyxp->zycp", A, G)
    return G.reshape(N ** 3, p)


def poisson_exact(b: np.ndarray, N: int, h: float) -> np.ndarray:
    """Exact solution of K v = b through the sine eigenbasis."""
    Phi = sine_basis(N)
    kap, mu = eigen_1d(N, h)
    lam = (kap[:, None, None] * mu[None, :, None] * mu[None, None, :]
           + mu[:, None, None] * kap[None, :, None] * mu[None, None, :]
           + mu[:, None, None] * mu[None, :, None] * kap[None, None, :])
    bh = _along_axes(np.asarray(b, dtype=np.float64).reshape(-1, 1), N, Phi)
    vh = bh / lam.reshape(-1, 1)
    return _along_axes(vh, N, Phi)[:, 0]


def mass_inverse(E: np.ndarray, N: int, h: float) -> np.ndarray:
    """G = M^{-1} E.  M = M1(x)M1(x)M1, so M^{-1} is the 1-D tridiagonal solve
    with M1 applied along each grid axis in turn (LAPACK banded solver)."""
    E = np.asarray(E, dtype=np.float64)
    squeeze = E.ndim == 1
    if squeeze:
        E = E[:, None]
    p = E.shape[1]
    ab = np.zeros((3, N))
    ab[0, 1:] = h / 6.0
    ab[1, :] = 4.0 * h / 6.0
    ab[2, :-1] = h / 6.0
    G = E.reshape(N, N, N, p)
    for axis in range(3):
        moved = np.moveaxis(G, axis, 0)
        shape = moved.shape
        sol = solve_banded((1, 1), ab, moved.reshape(N, -1))
        G = np.moveaxis(sol.reshape(shape), 0, axis)
    G = np.ascontiguousarray(G).reshape(N ** 3, p)
    return G[:, 0] if squeeze else G


def mass_inverse_sine(E: np.ndarray, N: int, h: float) -> np.ndarray:
    """M^{-1} E through the sine eigenbasis (independent cross-check)."""
    E = np.asarray(E, dtype=np.float64)
    squeeze = E.ndim == 1
    if squeeze:
        E = E[:, None]
    Phi = sine_basis(N)
    _, mu = eigen_1d(N, h)
    lam = (mu[:, None, None] * mu[None, :, None] * mu[None, None, :]).reshape(-1, 1)
    G = _along_axes(_along_axes(E, N, Phi) / lam, N, Phi)
    return G[:, 0] if squeeze else G


def generalized_eigs_closed_form(N: int, h: float) -> np.ndarray:
    """All eigenvalues of K v = lambda M v in ascending order:
    lambda_abc = sum over d in {a,b,c} of 6(1-cos t_d)/(h^2 (2+cos t_d))."""
    t = np.arange(1, N + 1) * np.pi / (N + 1)
    r = 6.0 * (1.0 - np.cos(t)) / (h * h * (2.0 + np.cos(t)))
    lam = r[:, None, None] + r[None, :, None] + r[None, None, :]
    return np.sort(lam.ravel())


def cg_solve(apply_A, b: np.ndarray, x0: np.ndarray | None, tol: float,
             maxit: int) -> tuple[np.ndarray, np.ndarray, int, bool]:
    """Plain conjugate gradients for an SPD operator (Hestenes-Stiefel),
    stopping when ||r||_2 <= tol ||b||_2.  Returns (x, r, iterations, ok)."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_A(x)
    bnorm = np.sqrt(b @ b)
    if bnorm == 0.0:
        return np.zeros_like(b), np.zeros_like(b), 0, True
    p = r.copy()
    rr = r @ r
    it = 0
    while np.sqrt(rr) > tol * bnorm:
        if it == maxit:
            return x, r, it, False
        q = apply_A(p)
        alpha = rr / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, r, it, True


def prolong_1d(Nc: int) -> np.ndarray:
    """1-D Q1 interpolation from Nc interior nodes (spacing h) to Nf = 2 Nc + 1
    (spacing h/2), zero Dirichlet values at both ends: fine node 2i+1 is
    coarse node i, fine node 2i lies halfway between coarse nodes i-1 and i.
    Returns the Nf x Nc matrix."""
    Nf = 2 * Nc + 1
    P = np.zeros((Nf, Nc))
    for i in range(Nc):
        P[2 * i + 1, i] = 1.0
        P[2 * i, i] += 0.5
        P[2 * i + 2, i] += 0.5
    return P


def prolong(X: np.ndarray, Nc: int) -> np.ndarray:
    """Uniform refinement of a Q1 field (Alg. AdpConOptM's projection of the
    coarse solution onto the next mesh): the fine nodal values of the same
    trilinear function, (P1 (x) P1 (x) P1) X, applied along each axis."""
    X = np.asarray(X, dtype=np.float64)
    squeeze = X.ndim == 1
    if squeeze:
        X = X[:, None]
    p = X.shape[1]
    P1 = prolong_1d(Nc)
    Nf = P1.shape[0]
    F = X.reshape(Nc, Nc, Nc, p)
    F = np.einsum("ai,ijkq->ajkq", P1, F)       # z
    F = np.einsum("bj,ajkq->abkq", P1, F)       # y
    F = np.einsum("ck,abkq->abcq", P1, F)       # x
    out = F.reshape(Nf ** 3, p)
    return out[:, 0] if squeeze else out
