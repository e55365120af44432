"""Gradient methods on the generalised Stiefel manifold X^T M X = I.

The paper minimises E(X) subject to X^T X = I (Eq. opt) and, for the finite
element model, uses y = B^{1/2} c to turn c^T B c = 1 into a unit sphere
(Eq. OFDFT-y).  The same substitution Y = M^{1/2} X maps X^T M X = I onto
the plain Stiefel manifold; every formula below is the paper's formula in Y
written back in X, so that M^{1/2} is never formed:

  gradient  (Eq. def-nablaE)  D = M^{-1} E_X - X (E_X^T X),  ||D||^2_M = tr(D^T M D)
  QR        (Eq. QR, Alg. ChQR)  Y = X - tau D,  Y^T M Y = L L^T,  X+ = Y L^{-T}
  Cayley    (Eq. WY3)  U = [M^{-1}E_X, X],  V^T U = [[X^T E_X, X^T M X], [-E_X^T M^{-1} E_X, -E_X^T X]],
            V^T Y = [X^T M X; -E_X^T X],  X+ = X - tau U (I + tau/2 V^T U)^{-1} V^T Y
  BB        (Eq. bb-1)  S = X_k - X_{k-1}, Y = D_k - D_{k-1}, traces in the M inner product
  search    (Eq. NMLS-Armijo)  E(X_k(tau)) <= C_k - rho1 tau ||D_k||^2_M,  tau = tau_BB delta^h
            Q_{k+1} = eta Q_k + 1,  C_{k+1} = (eta Q_k C_k + E(X_{k+1})) / Q_{k+1}
  driver    Alg. ConOptM.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.linalg import cholesky, solve_triangular, solve, sqrtm

from . import fe
from .energy import Model, Evaluation, evaluate


@dataclass
class Point:
    """Everything the iteration needs at one feasible X."""
    X: np.ndarray
    MX: np.ndarray
    ev: Evaluation
    G: np.ndarray          # M^{-1} E_X
    S: np.ndarray          # E_X^T X
    D: np.ndarray          # projected gradient
    MD: np.ndarray         # M D
    dnorm2: float          # ||D||_M^2

    @property
    def E(self) -> float:
        return self.ev.E

    @property
    def dnorm(self) -> float:
        return math.sqrt(max(self.dnorm2, 0.0))


def m_orthonormalize(model: Model, X: np.ndarray, passes: int = 2) -> np.ndarray:
    """Cholesky QR in the M inner product (Alg. ChQR with Y^T M Y), repeated
    `passes` times: O = X^T M X = L L^T, X <- X L^{-T}."""
    X = np.array(X, dtype=np.float64)
    for _ in range(passes):
        O = X.T @ model.apply_M(X)
        Lc = cholesky(0.5 * (O + O.T), lower=True)
        X = solve_triangular(Lc, X.T, lower=True).T
    return X


def ortho_error(model: Model, X: np.ndarray, MX: np.ndarray | None = None) -> float:
    """||X^T M X - I||_F."""
    if MX is None:
        MX = model.apply_M(X)
    return float(np.linalg.norm(X.T @ MX - np.eye(X.shape[1])))


def project(model: Model, X: np.ndarray, ev: Evaluation) -> Point:
    """Riemannian gradient in the M metric (Eq. def-nablaE in Y = M^{1/2} X)."""
    N, h = model.N, model.h
    G = model.mass_inverse(ev.EX)
    S = ev.EX.T @ X
    D = G - X @ S
    MD = model.apply_M(D)
    MX = model.apply_M(X)
    return Point(X=X, MX=MX, ev=ev, G=G, S=S, D=D, MD=MD, dnorm2=float(np.sum(D * MD)))


def point_at(model: Model, X: np.ndarray, v_guess=None) -> Point:
    return project(model, X, evaluate(model, X, v_guess))


def retract_qr(model: Model, pt: Point, tau: float) -> np.ndarray:
    """Eq. QR with Alg. ChQR: Y = X - tau D; Y^T M Y = L L^T; Q = Y L^{-T}."""
    Y = pt.X - tau * pt.D
    R = Y.T @ model.apply_M(Y)
    Lc = cholesky(0.5 * (R + R.T), lower=True)
    return solve_triangular(Lc, Y.T, lower=True).T


def cayley_blocks(model: Model, pt: Point):
    """U, V^T U and V^T Y of Eq. WY3 written in X coordinates."""
    X, EX, G = pt.X, pt.ev.EX, pt.G
    O = X.T @ pt.MX
    S = pt.S                                    # E_X^T X
    A = X.T @ EX                                # X^T E_X
    B = EX.T @ G                                # E_X^T M^{-1} E_X
    VU = np.block([[A, O], [-B, -S]])
    VY = np.vstack([O, -S])
    U = np.hstack([G, X])
    return U, VU, VY


def retract_cayley(model: Model, pt: Point, tau: float) -> np.ndarray:
    """Eq. WY3: X+ = X - tau U (I + tau/2 V^T U)^{-1} V^T Y."""
    U, VU, VY = cayley_blocks(model, pt)
    P = solve(np.eye(VU.shape[0]) + 0.5 * tau * VU, VY)
    return pt.X - tau * (U @ P)


def retract_cayley_dense(model: Model, pt: Point, tau: float) -> np.ndarray:
    """Eq. WY1 with the dense n x n skew matrix W, in Y = M^{1/2} X (tiny n)."""
    M = model.dense_M()
    Mh = np.real(sqrtm(M))
    Mmh = np.linalg.inv(Mh)
    Y = Mh @ pt.X
    EY = Mmh @ pt.ev.EX
    W = EY @ Y.T - Y @ EY.T
    I = np.eye(W.shape[0])
    Yn = solve(I + 0.5 * tau * W, (I - 0.5 * tau * W) @ Y)
    return Mmh @ Yn


def retract_cayley_p1(model: Model, pt: Point, tau: float) -> np.ndarray:
    """Eq. WY-1d for p = 1 in Y coordinates: with x = Y, a = E_Y,
    x+ = x - beta1 a - beta2 x; inner products a^T x = E_X^T X,
    a^T a = E_X^T M^{-1} E_X, x^T x = X^T M X, and M^{-1/2} a = M^{-1} E_X."""
    x, g = pt.X[:, 0], pt.G[:, 0]
    ax = float(pt.ev.EX[:, 0] @ x)
    aa = float(pt.ev.EX[:, 0] @ g)
    xx = float(x @ pt.MX[:, 0])
    t2 = (0.5 * tau) ** 2
    den = 1.0 - t2 * ax * ax + t2 * aa * xx
    beta1 = tau * xx / den
    beta2 = -tau * (ax + 0.5 * tau * (ax * ax - aa * xx)) / den
    return (x - beta1 * g - beta2 * x)[:, None]


@dataclass
class Options:
    """Parameters of Alg. ConOptM (the paper gives no values; these are the
    readings recorded with the results)."""
    retraction: str = "qr"
    gtol: float = 1e-6
    maxit: int = 300
    tau0: float = 1e-3
    rho1: float = 1e-4
    delta: float = 0.1
    eta: float = 0.85
    tau_min: float = 1e-10
    tau_max: float = 1e10
    max_backtrack: int = 10
    ortho_tol: float = 1e-12
    # Rounding slack of the Armijo test: when set, a trial is also accepted
    # if its energy exceeds C - rho1 tau ||D||^2 by at most
    # 4 eps sum |E_parts| (eps = 2^-52), the rounding of the energy sums.
    # In exact arithmetic the test of Eq. NMLS-Armijo always accepts a small
    # enough step; in FP64 near convergence the required decrease falls below
    # that rounding and the exact test backtracks at random.  Off by default.
    armijo_slack: bool = False


@dataclass
class Result:
    X: np.ndarray
    E: float
    parts: dict
    dnorm: float
    iters: int
    converged: bool
    history: list = field(default_factory=list)
    point: Point | None = None


def bb_traces(model: Model, cur: Point, prev: Point) -> tuple[float, float, float]:
    """tr(S^T M S), tr(S^T M Y), tr(Y^T M Y) with S = X_k - X_{k-1} and
    Y = D_k - D_{k-1} (Eq. bb-1 in the M inner product)."""
    dX = cur.X - prev.X
    dMX = cur.MX - prev.MX
    dD = cur.D - prev.D
    dMD = cur.MD - prev.MD
    return float(np.sum(dX * dMX)), float(np.sum(dX * dMD)), float(np.sum(dD * dMD))


def bb_step(k: int, ss: float, sy: float, yy: float, opt: Options) -> float:
    """tau_{k,1} = ss/|sy| on odd k, tau_{k,2} = |sy|/yy on even k; reset to
    tau0 when the quotient is not a positive finite number, then clamp."""
    if k % 2 == 1:
        num, den = ss, abs(sy)
    else:
        num, den = abs(sy), yy
    if not (den > 0.0) or not math.isfinite(num) or not math.isfinite(den):
        return opt.tau0
    tau = num / den
    if not math.isfinite(tau) or tau <= 0.0:
        return opt.tau0
    return min(max(tau, opt.tau_min), opt.tau_max)


def armijo_slack(parts: dict, opt: Options) -> float:
    """4 eps sum |E_parts| when opt.armijo_slack is set, else 0."""
    if not opt.armijo_slack:
        return 0.0
    return 4.0 * 2.220446049250313e-16 * sum(abs(v) for v in parts.values())


def minimize(model: Model, X0: np.ndarray, opt: Options | None = None,
             orthonormalize: bool = True, callback=None) -> Result:
    """Alg. ConOptM.  X0 is M-orthonormalised first unless told otherwise."""
    opt = opt or Options()
    retract = retract_qr if opt.retraction == "qr" else retract_cayley
    if opt.retraction != "qr" and model.p == 1:
        retract = retract_cayley_p1              # Lemma 3.1 (3): no 2 x 2 solve
    X = m_orthonormalize(model, X0) if orthonormalize else np.array(X0, dtype=np.float64)
    cur = point_at(model, X)
    C, Q = cur.E, 1.0
    prev = None
    history = []
    k = 0
    while cur.dnorm > opt.gtol and k < opt.maxit:
        if prev is None:
            tau = opt.tau0
        else:
            tau = bb_step(k, *bb_traces(model, cur, prev), opt)
        h = 0
        while True:
            Xn = retract(model, cur, tau)
            trial = point_at(model, Xn, cur.ev.vH)
            bound = C - opt.rho1 * tau * cur.dnorm2
            slack = armijo_slack(trial.ev.parts, opt)
            ok = trial.E <= bound + slack
            if ok or h == opt.max_backtrack:
                break
            tau *= opt.delta
            h += 1
        Qn = opt.eta * Q + 1.0
        C = (opt.eta * Q * C + trial.E) / Qn
        Q = Qn
        if not ok:
            # the last trial is taken without meeting the test: the
            # nonmonotone reference restarts at its energy (C_k >= E_k holds)
            C, Q = trial.E, 1.0
        oerr = ortho_error(model, trial.X, trial.MX)
        if opt.retraction != "qr" and oerr > opt.ortho_tol:
            trial = point_at(model, m_orthonormalize(model, trial.X, passes=1), cur.ev.vH)
        history.append({"k": k, "E": trial.E, "dnorm": trial.dnorm, "tau": tau, "h": h,
                        "C": C, "Q": Q, "ortho": oerr, "cg": trial.ev.cg_iters,
                        "forced": not ok, "excess": trial.E - bound, "slack": slack})
        prev, cur = cur, trial
        k += 1
        if callback is not None:
            callback(k, cur)
    return Result(X=cur.X, E=cur.E, parts=cur.ev.parts, dnorm=cur.dnorm, iters=k,
                  converged=cur.dnorm <= opt.gtol, history=history, point=cur)


def refine_levels(N: int, levels: int) -> list[int]:
    """Grids of a uniform refinement ending at N: N_l = (N+1) / 2^(levels-1-l) - 1."""
    if levels < 1 or (N + 1) % (1 << (levels - 1)) != 0:
        raise ValueError("N + 1 must be divisible by 2^(levels - 1)")
    out = [(N + 1) // (1 << (levels - 1 - l)) - 1 for l in range(levels)]
    if out[0] < 2:
        raise ValueError("coarsest grid below 2 nodes per edge")
    return out


def minimize_refine(model: Model, X0: np.ndarray, levels: int, opt: Options | None = None,
                    coarse_gtol: float = 1e-3) -> list[Result]:
    """Alg. AdpConOptM with uniform refinement and a fixed number of levels:
    Alg. ConOptM on each grid of refine_levels(model.N, levels) in turn, the
    coarser levels to coarse_gtol, each level started from the Q1
    interpolant of the previous level's solution (M-orthonormalised on the
    new grid).  X0 is the initial block on the coarsest grid.  Returns the
    result of every level (the last one on model's own grid)."""
    from dataclasses import replace
    opt = opt or Options()
    grids = refine_levels(model.N, levels)
    results = []
    X = X0
    for l, Nl in enumerate(grids):
        m = replace(model, N=Nl, _vext=None)
        o = replace(opt, gtol=opt.gtol if l == levels - 1 else coarse_gtol)
        r = minimize(m, X, o)
        results.append(r)
        if l < levels - 1:
            X = fe.prolong(r.X, Nl)
    return results

