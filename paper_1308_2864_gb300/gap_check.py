"""Levels around the Fermi level of a converged system: the occupied orbital
energies (the spectrum of Lambda = sym(X^T E_X) / 2f at the returned block,
the Lagrange multipliers of Eq. disKS) and the lowest unoccupied levels of
the Kohn-Sham operator H = K/2 + h^3 Diag(V_eff) at the converged density,
found by LOBPCG in the M metric with the occupied block as a constraint.

The gap between them decides how fast a gradient method on the Stiefel
manifold converges (the paper's Sec. 5 discusses its systems' gaps): the
Hessian of the energy along a rotation of occupied orbital i into
unoccupied level a scales like eps_a - eps_i, so a vanishing gap makes the
BB iteration crawl.

  python -m paper_1308_2864_gb300.gap_check --config c2 [--k 8] [--maxit 200000]

Runs the mixed-precision solve to gtol (or maxit), then LOBPCG (scipy) with
H and M applied by the library's FP64 stencil kernels on the GPU and
(K/2 + sigma M)^{-1} as preconditioner, diagonal in the sine basis that
diagonalises both Q1 operators (applied with torch on the GPU).  Prints one
JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None) -> int:
    import numpy as np
    import scipy.sparse.linalg as sla
    import torch

    import ks_inputs as ki
    import paper_1308_2864_gb300 as ks

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--config", default="c2", choices=sorted(ki.CONFIGS))
    ap.add_argument("--k", type=int, default=8, help="unoccupied levels to find")
    ap.add_argument("--maxit", type=int, default=200000)
    ap.add_argument("--gtol", type=float, default=1e-6)
    ap.add_argument("--sigma", type=float, default=8.0, help="shift of the preconditioner (Ha)")
    a = ap.parse_args(argv)

    s = ki.CONFIGS[a.config]()
    P = ks.Problem.from_system(s)
    P.set_fp64_emulation(1)
    X = torch.from_numpy(np.ascontiguousarray(s.x0())).cuda()
    t0 = time.perf_counter()
    r = P.minimize(X, retraction=s.retraction, gtol=a.gtol, maxit=a.maxit, precision="mixed")
    torch.cuda.synchronize()
    solve_s = time.perf_counter() - t0
    N, n, f, k = s.N, s.n, s.occ, a.k
    h = s.L / (N + 1)
    rho = P.step_density(X)
    vH, res, _ = P.step_hartree(rho)
    veff, _ = P.step_potential(rho, vH, res)
    EX, _, _ = P.step_hamiltonian(X, veff)
    Lam = (X.T @ EX).cpu().numpy()
    occ = np.linalg.eigvalsh(0.5 * (Lam + Lam.T)) / (2.0 * f)

    sk = ki.CONFIGS[a.config]()
    sk.p = k
    Pk = ks.Problem.from_system(sk)
    j = torch.arange(1, N + 1, dtype=torch.float64, device="cuda")
    th = j * math.pi / (N + 1)
    Phi = math.sqrt(2.0 / (N + 1)) * torch.sin(torch.outer(j, j) * math.pi / (N + 1))
    kap = (2.0 / h) * (1 - torch.cos(th))
    mu = (h / 3.0) * (2 + torch.cos(th))
    lamK = (kap[:, None, None] * mu[None, :, None] * mu[None, None, :]
            + mu[:, None, None] * kap[None, :, None] * mu[None, None, :]
            + mu[:, None, None] * mu[None, :, None] * kap[None, None, :])
    lamM = mu[:, None, None] * mu[None, :, None] * mu[None, None, :]
    den = 0.5 * lamK + a.sigma * lamM

    def sine3(V):
        G = V.reshape(N, N, N, -1)
        G = torch.einsum("az,zyxm->ayxm", Phi, G)
        G = torch.einsum("by,ayxm->abxm", Phi, G)
        return torch.einsum("cx,abxm->abcm", Phi, G)

    def blockwise(fn, V):
        V = np.asarray(V, dtype=np.float64)
        one = V.ndim == 1
        V2 = V[:, None] if one else V
        m = V2.shape[1]
        pad = (-m) % k
        Vt = torch.from_numpy(np.ascontiguousarray(V2)).cuda()
        if pad:
            Vt = torch.cat([Vt, torch.zeros(n, pad, dtype=torch.float64, device="cuda")], dim=1)
        out = torch.cat([fn(Vt[:, i:i + k].contiguous()) for i in range(0, Vt.shape[1], k)],
                        dim=1)[:, :m].cpu().numpy()
        return out[:, 0] if one else out

    def h_op(V):   # E_X of the k-wide problem at fixed V_eff is 2f H V
        return blockwise(lambda B: Pk.step_hamiltonian(B, veff, want_mx=False)[0] / (2.0 * f), V)

    def m_op(V):
        return blockwise(lambda B: Pk.step_mass(B), V)

    def t_op(V):
        return blockwise(lambda B: sine3(sine3(B).div(den[..., None]).reshape(n, -1))
                         .reshape(n, -1), V)

    A = sla.LinearOperator((n, n), matvec=h_op, matmat=h_op, dtype=np.float64)
    Mm = sla.LinearOperator((n, n), matvec=m_op, matmat=m_op, dtype=np.float64)
    T = sla.LinearOperator((n, n), matvec=t_op, matmat=t_op, dtype=np.float64)
    V0 = np.random.default_rng(0).standard_normal((n, k))
    t1 = time.perf_counter()
    w, _, hist = sla.lobpcg(A, V0, B=Mm, M=T, Y=X.cpu().numpy(), tol=1e-7, maxiter=400,
                            largest=False, retResidualNormsHistory=True)
    w = np.sort(w)
    print(json.dumps({
        "config": a.config, "solve": {"E": r["E"], "gradnorm": r["gradnorm"], "iters": r["iters"],
                                      "seconds": solve_s},
        "occupied_eps": occ.tolist(), "homo": float(occ[-1]),
        "lowest_unoccupied_eps": w.tolist(), "lumo": float(w[0]),
        "gap_Ha": float(w[0] - occ[-1]),
        "lobpcg_iters": len(hist), "lobpcg_max_residual": float(np.max(hist[-1])),
        "lobpcg_seconds": time.perf_counter() - t1}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
