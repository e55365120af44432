"""The discrete Kohn-Sham total energy and its derivative.

Continuous functional: Eq. EKS, E = T_KS + E_H + E_xc + E_ext + E_II
(Sec. 2.1).  Discrete form: Sec. 2.3 gives
  E(X) = 1/2 tr(X^T L X) + tr(X^T E X) + 1/2 rho^T L^+ rho + rho^T eps_xc(rho),
  rho(X) = diag(X X^T),  E_X = H(X) X.
Restated for Q1 elements with occupation f (where the paper is silent, the
choices are stated here):

  rho_k  = f sum_i X_ki^2                               (nodal density)
  E(X)   = (f/2) tr(X^T K X)                              kinetic
         + h^3 sum_k Vext_k rho_k                          external
         + 1/2 h^3 sum_k vH_k rho_k,  K vH = 4 pi h^3 rho  Hartree
         + h^3 sum_k rho_k eps_xc(rho_k)                   exchange-correlation
         + E_II                                            ion-ion
  E_X    = f K X + 2 f h^3 Diag(Vext + vH + v_xc) X,  v_xc = d(rho eps_xc)/d rho

E_X is the exact derivative of E (the paper's H(X)X up to the factor 2f of
its own normalisation; the finite-difference test pins this).

Orbital-free model (Sec. 2.2, Eq. TFW and Eq. OFeng; discretised as
Eq. disOFinf with c^T M c = 1): one amplitude c = X (p = 1) carries all
f = N_e electrons, rho_k = f c_k^2, and the kinetic term is the TFW density
functional C_TF T_TF + mu T_vW.  With rho = phi^2 the von Weizsaecker term
(1/8) int |grad rho|^2 / rho equals (1/2) int |grad phi|^2, which for the Q1
interpolant of phi = sqrt(f) c is (f/2) c^T K c; the Thomas-Fermi term uses
the same nodal quadrature as E_xc:

  E(c)   = mu (f/2) c^T K c + h^3 sum_k C_TF rho_k^(5/3)   kinetic (TFW)
         + external + Hartree + xc + ion-ion                as above
  E_c    = mu f K c + 2 f h^3 Diag(Vext + vH + v_xc + v_TF) c,
  v_TF   = (5/3) C_TF rho^(2/3),  C_TF = (3/10) (3 pi^2)^(2/3).

When the Hartree potential comes from an inexact solve with residual
r = 4 pi h^3 rho - K vH, the energy uses the variational form
E_H = 1/2 h^3 rho^T vH + vH^T r / (8 pi), which equals the definition when
r = 0 and differs from the exact value only to second order in the solve
error.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.special import erf

from . import fe

XC_SLATER = 0
XC_SLATER_PZ81 = 1
MASS_CONSISTENT = 0     # M = M1 (x) M1 (x) M1, the Q1 mass matrix
MASS_LUMPED = 1         # M = h^3 I, its row sums (mass lumping)
KIN_ORBITALS = 0        # (f/2) tr(X^T K X), Eq. EKS
KIN_TFW = 1             # Thomas-Fermi-von Weizsaecker, Eq. TFW (p = 1)
C_TF = 0.3 * (3.0 * math.pi ** 2) ** (2.0 / 3.0)

# Perdew-Zunger (1981) parametrisation of the Ceperley-Alder correlation
# energy, unpolarised gas, in hartree.  gamma, beta1, beta2 (r_s >= 1) and
# A, B (r_s < 1) are the published values.  The published C = 0.0020 and
# D = -0.0116 are rounded values of the coefficients that make eps_c and
# d eps_c / d r_s continuous at r_s = 1; rounded, they leave a 3.2e-5 Ha jump
# in eps_c there, which makes the discrete energy discontinuous.  C and D are
# therefore taken from the two continuity conditions:
#   B + D = gamma / (1 + beta1 + beta2)
#   A + C + D = -gamma (beta1/2 + beta2) / (1 + beta1 + beta2)^2
PZ_GAMMA, PZ_BETA1, PZ_BETA2 = -0.1423, 1.0529, 0.3334
PZ_A, PZ_B = 0.0311, -0.048
_PZ_DEN1 = 1.0 + PZ_BETA1 + PZ_BETA2
PZ_D = PZ_GAMMA / _PZ_DEN1 - PZ_B
PZ_C = -PZ_GAMMA * (0.5 * PZ_BETA1 + PZ_BETA2) / (_PZ_DEN1 * _PZ_DEN1) - PZ_A - PZ_D
RHO_FLOOR = 1e-30


def node_coords(N: int, h: float) -> np.ndarray:
    """(n, 3) coordinates (x, y, z) of the interior nodes, flat order k."""
    g = (np.arange(N) + 1.0) * h
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def v_ext(N: int, h: float, atoms: np.ndarray, Z: np.ndarray, rc: float) -> np.ndarray:
    """Local pseudo-atom potential sum_a -Z_a erf(|r-R_a|/rc)/|r-R_a|; at
    |r-R_a| < 1e-6 the series -Z_a (2/(sqrt(pi) rc)) (1 - r^2/(3 rc^2))."""
    r_nodes = node_coords(N, h)
    V = np.zeros(N ** 3)
    for R, Za in zip(atoms, Z):
        r = np.linalg.norm(r_nodes - R[None, :], axis=1)
        small = r < 1e-6
        rs = np.where(small, 1.0, r)
        V += np.where(small,
                      -Za * (2.0 / (math.sqrt(math.pi) * rc)) * (1.0 - r * r / (3.0 * rc * rc)),
                      -Za * erf(rs / rc) / rs)
    return V


def e_ii(atoms: np.ndarray, Z: np.ndarray) -> float:
    """Nuclear repulsion 1/2 sum_{i != j} Z_i Z_j / |R_i - R_j| (Sec. 2.1)."""
    e = 0.0
    for i in range(len(Z)):
        for j in range(len(Z)):
            if i != j:
                e += 0.5 * Z[i] * Z[j] / np.linalg.norm(atoms[i] - atoms[j])
    return e


def slater(rho: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Slater (Dirac) exchange: eps_x = -(3/4)(3/pi)^(1/3) rho^(1/3),
    v_x = d(rho eps_x)/d rho = -(3/pi)^(1/3) rho^(1/3)."""
    c = (3.0 / math.pi) ** (1.0 / 3.0)
    r13 = np.cbrt(rho)
    return -0.75 * c * r13, -c * r13


def pz81(rho: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Perdew-Zunger correlation, rs = (3/(4 pi rho))^(1/3):
      rs >= 1: eps_c = gamma / (1 + beta1 sqrt(rs) + beta2 rs)
      rs <  1: eps_c = A ln rs + B + C rs ln rs + D rs
    and v_c = eps_c - (rs/3) d eps_c / d rs."""
    rs = np.cbrt(3.0 / (4.0 * math.pi * rho))
    hi = rs >= 1.0
    srs = np.sqrt(rs)
    den = 1.0 + PZ_BETA1 * srs + PZ_BETA2 * rs
    eps_hi = PZ_GAMMA / den
    deps_hi = -PZ_GAMMA * (0.5 * PZ_BETA1 / srs + PZ_BETA2) / (den * den)
    lrs = np.log(rs)
    eps_lo = PZ_A * lrs + PZ_B + PZ_C * rs * lrs + PZ_D * rs
    deps_lo = PZ_A / rs + PZ_C * (lrs + 1.0) + PZ_D
    eps = np.where(hi, eps_hi, eps_lo)
    deps = np.where(hi, deps_hi, deps_lo)
    return eps, eps - (rs / 3.0) * deps


def thomas_fermi(rho: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Thomas-Fermi kinetic energy per unit volume C_TF rho^(5/3) (the
    integrand of T_TF in Eq. TFW, with its constant C_TF) and its derivative
    v_TF = (5/3) C_TF rho^(2/3); both 0 below RHO_FLOOR."""
    rho = np.asarray(rho, dtype=np.float64)
    ok = rho >= RHO_FLOOR
    r = np.where(ok, rho, 1.0)
    r23 = np.cbrt(r) ** 2
    e = C_TF * r * r23
    v = (5.0 / 3.0) * C_TF * r23
    return np.where(ok, e, 0.0), np.where(ok, v, 0.0)


def lda(rho: np.ndarray, xc: int) -> tuple[np.ndarray, np.ndarray]:
    """LDA energy per electron eps_xc and potential v_xc; both are set to 0
    where rho < 1e-30."""
    rho = np.asarray(rho, dtype=np.float64)
    ok = rho >= RHO_FLOOR
    r = np.where(ok, rho, 1.0)
    eps, v = slater(r)
    if xc == XC_SLATER_PZ81:
        ec, vc = pz81(r)
        eps, v = eps + ec, v + vc
    return np.where(ok, eps, 0.0), np.where(ok, v, 0.0)


@dataclass
class Model:
    """A discretised KS system.  The switches drop terms for the pins
    (e.g. V = 0 gives the closed-form Laplacian problem)."""
    N: int
    L: float
    atoms: np.ndarray
    Z: np.ndarray
    p: int
    xc: int = XC_SLATER_PZ81
    rc: float = 0.5
    occ: float = 2.0
    mass: int = MASS_CONSISTENT
    kinetic: int = KIN_ORBITALS
    mu: float = 1.0                 # von Weizsaecker weight (KIN_TFW)
    use_tf: bool = True             # KIN_TFW: include the Thomas-Fermi term
    use_ext: bool = True
    use_hartree: bool = True
    use_xc: bool = True
    use_eii: bool = True
    poisson: str = "exact"          # "exact" (sine basis) or "cg"
    cg_tol: float = 1e-10
    cg_maxit: int = 10_000
    _vext: np.ndarray | None = field(default=None, repr=False)

    @property
    def h(self) -> float:
        return self.L / (self.N + 1)

    @property
    def n(self) -> int:
        return self.N ** 3

    @classmethod
    def from_system(cls, s, **kw) -> "Model":
        kw.setdefault("kinetic", getattr(s, "kinetic", KIN_ORBITALS))
        kw.setdefault("mass", getattr(s, "mass", MASS_CONSISTENT))
        kw.setdefault("mu", getattr(s, "mu", 1.0))
        return cls(N=s.N, L=s.L, atoms=np.asarray(s.atoms), Z=np.asarray(s.Z), p=s.p,
                   xc=s.xc, rc=s.rc, occ=s.occ, **kw)

    def __post_init__(self):
        if self.kinetic == KIN_TFW and self.p != 1:
            raise ValueError("the TFW kinetic functional takes one amplitude (p = 1)")

    def apply_M(self, X: np.ndarray) -> np.ndarray:
        """M X: the Q1 mass matrix, or its row sums h^3 (lumped)."""
        if self.mass == MASS_LUMPED:
            return self.h ** 3 * np.asarray(X, dtype=np.float64)
        return fe.apply_M(X, self.N, self.h)

    def mass_inverse(self, X: np.ndarray) -> np.ndarray:
        if self.mass == MASS_LUMPED:
            return np.asarray(X, dtype=np.float64) / self.h ** 3
        return fe.mass_inverse(X, self.N, self.h)

    def dense_M(self) -> np.ndarray:
        if self.mass == MASS_LUMPED:
            return self.h ** 3 * np.eye(self.n)
        return fe.dense_K_M(self.N, self.h)[1]

    @property
    def kin_weight(self) -> float:
        """Factor of (f/2) tr(X^T K X): 1 for orbitals, mu for TFW."""
        return self.mu if self.kinetic == KIN_TFW else 1.0

    def vext(self) -> np.ndarray:
        if self._vext is None:
            self._vext = (v_ext(self.N, self.h, self.atoms, self.Z, self.rc)
                          if self.use_ext else np.zeros(self.n))
        return self._vext

    def eii(self) -> float:
        return e_ii(self.atoms, self.Z) if (self.use_eii and self.use_ext) else 0.0


@dataclass
class Evaluation:
    E: float
    parts: dict                      # kinetic, external, hartree, xc, ion
    EX: np.ndarray                   # dE/dX
    rho: np.ndarray
    vH: np.ndarray
    veff: np.ndarray
    cg_iters: int = 0


def density(X: np.ndarray, occ: float) -> np.ndarray:
    """rho = f diag(X X^T) (Sec. 2.3, with occupation f)."""
    return occ * np.einsum("ki,ki->k", X, X)


def hartree(model: Model, rho: np.ndarray, v_guess: np.ndarray | None = None):
    """Solve K vH = 4 pi h^3 rho.  Returns (vH, residual, iterations)."""
    h, N = model.h, model.N
    b = 4.0 * math.pi * h ** 3 * rho
    if model.poisson == "exact":
        return fe.poisson_exact(b, N, h), np.zeros_like(b), 0
    vH, r, it, ok = fe.cg_solve(lambda v: fe.apply_K(v, N, h), b, v_guess,
                                model.cg_tol, model.cg_maxit)
    if not ok:
        raise RuntimeError("Hartree CG did not converge")
    return vH, r, it


def evaluate(model: Model, X: np.ndarray, v_guess: np.ndarray | None = None) -> Evaluation:
    """Total energy and its derivative E_X at X (not necessarily feasible)."""
    N, h, f = model.N, model.h, model.occ
    h3 = h ** 3
    X = np.asarray(X, dtype=np.float64)
    rho = density(X, f)
    KX = fe.apply_K(X, N, h)
    w = model.kin_weight
    e_kin = 0.5 * f * w * float(np.sum(X * KX))
    vext = model.vext()
    e_ext = h3 * float(vext @ rho)
    veff = vext.copy()
    if model.kinetic == KIN_TFW and model.use_tf:
        etf, vtf = thomas_fermi(rho)
        e_kin += h3 * float(np.sum(etf))
        veff += vtf
    vH = np.zeros_like(rho)
    e_h = 0.0
    it = 0
    if model.use_hartree:
        vH, r, it = hartree(model, rho, v_guess)
        e_h = 0.5 * h3 * float(vH @ rho) + float(vH @ r) / (8.0 * math.pi)
        veff += vH
    e_xc = 0.0
    if model.use_xc:
        eps, vxc = lda(rho, model.xc)
        e_xc = h3 * float(rho @ eps)
        veff += vxc
    e_ion = model.eii()
    EX = w * f * KX + 2.0 * f * h3 * veff[:, None] * X
    parts = {"kinetic": e_kin, "external": e_ext, "hartree": e_h, "xc": e_xc, "ion": e_ion}
    return Evaluation(E=e_kin + e_ext + e_h + e_xc + e_ion, parts=parts, EX=EX,
                      rho=rho, vH=vH, veff=veff, cg_iters=it)
