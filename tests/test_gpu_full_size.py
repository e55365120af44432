"""Parity at the full sizes of the workloads, in the launch configuration
the benchmark times: the 64^3 / p = 64 system (every entry, the oracle
computes it in seconds) and the 128^3 / p = 512 system (the energy terms the
oracle computes from the full density, and E_X on sampled nodes, each from
its 27-node neighbourhood)."""
import math

import numpy as np
import pytest

import ks_inputs as ki
from oracle import energy as oe
from oracle import fe as ofe
from oracle import stiefel as ost

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel_err(got, want):
    return float(np.abs(np.asarray(got) - np.asarray(want)).max() / max(np.abs(want).max(), 1e-300))


def test_c2_full_size_energy_gradient_and_step():
    import paper_1308_2864_gb300 as ks
    s = ki.config_c2()
    model = oe.Model.from_system(s)
    X = ost.m_orthonormalize(model, s.x0())
    ref = oe.evaluate(model, X)
    pt = ost.project(model, X, ref)
    P = ks.Problem.from_system(s)
    E, EX, D, g = P.energy_grad(dev(X), want_d=True)
    assert E == pytest.approx(ref.E, rel=1e-11)
    assert rel_err(EX.cpu().numpy(), ref.EX) <= 1e-10
    assert rel_err(D.cpu().numpy(), pt.D) <= 1e-9
    parts = P.energy_parts()
    for got, key in zip(parts, ["kinetic", "external", "hartree", "xc", "ion"]):
        assert got == pytest.approx(ref.parts[key], rel=1e-10, abs=1e-9)
    Xn = P.retract(ks.KS_QR, dev(X), EX, 0.05).cpu().numpy()
    assert rel_err(Xn, ost.retract_qr(model, pt, 0.05)) <= 1e-9


def _kx_at(X, N, h, k):
    """(K X)_k from the 3 x 3 x 3 neighbourhood of node k (zero outside the
    grid, as the Dirichlet condition has it), with the oracle's stencil."""
    p = X.shape[1]
    iz, rem = divmod(k, N * N)
    iy, ix = divmod(rem, N)
    sub = np.zeros((27, p))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                z, y, x = iz + dz - 1, iy + dy - 1, ix + dx - 1
                if 0 <= z < N and 0 <= y < N and 0 <= x < N:
                    sub[(dz * 3 + dy) * 3 + dx] = X[(z * N + y) * N + x]
    return ofe.apply_K(sub, 3, h)[13]


def test_c3_full_size_energy_terms_and_sampled_gradient():
    import paper_1308_2864_gb300 as ks
    free, _ = torch.cuda.mem_get_info()
    if free < 135 * 2 ** 30:
        pytest.skip("needs about 130 GB of free device memory")
    s = ki.config_c3()
    model = oe.Model.from_system(s)
    N, h, f = model.N, model.h, model.occ
    h3 = h ** 3
    X = s.x0()
    P = ks.Problem.from_system(s)
    Xd = dev(X)
    E, EX, _, _ = P.energy_grad(Xd)
    parts = P.energy_parts()
    del Xd
    # the density terms from the oracle's full density
    rho = oe.density(X, f)
    vext = model.vext()
    vH = ofe.poisson_exact(4.0 * math.pi * h3 * rho, N, h)
    eps, vxc = oe.lda(rho, model.xc)
    assert parts[1] == pytest.approx(h3 * float(vext @ rho), rel=1e-11)
    assert parts[2] == pytest.approx(0.5 * h3 * float(vH @ rho), rel=1e-9)
    assert parts[3] == pytest.approx(h3 * float(rho @ eps), rel=1e-11)
    assert parts[4] == pytest.approx(model.eii(), rel=1e-13)
    veff = vext + vH + vxc
    # E_X on sampled nodes: corners, faces and seeded interior nodes
    rng = np.random.default_rng(2024)
    nodes = [0, N - 1, N * N - 1, N ** 3 - 1, (N // 2) * N * N + (N // 2) * N + N // 2]
    nodes += [int(k) for k in rng.integers(0, N ** 3, 40)]
    got = EX[torch.tensor(nodes, device="cuda")].cpu().numpy()
    for row, k in zip(got, nodes):
        want = f * _kx_at(X, N, h, k) + 2.0 * f * h3 * veff[k] * X[k]
        assert rel_err(row, want) <= 1e-9, f"node {k}"
