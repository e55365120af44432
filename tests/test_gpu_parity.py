"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on
the same seeded inputs.  Deterministic steps are compared element by element
at 1e-12 relative; the Hartree CG against its own tolerance; the full
minimisation on final energies (1e-8 Ha) and invariants."""
import math

import numpy as np
import pytest

import ks_inputs as ki
from oracle import energy as oe
from oracle import fe as ofe
from oracle import stiefel as ost

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-12


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def assert_rel(got, want, rel=REL, what=""):
    got, want = np.asarray(got), np.asarray(want)
    scale = max(np.abs(want).max(), 1e-300)
    err = np.abs(got - want).max() / scale
    assert err <= rel, f"{what}: max error {err:.3e} relative to max |want| > {rel:.1e}"


def make(system, **kw):
    import paper_1308_2864_gb300 as ks
    return ks.Problem.from_system(system, **kw)


# ragged sizes: n = 13^3 is not a multiple of any tile; p = 70 spans two
# 64-wide tiles with a ragged tail; p = 5 is below a warp.
SMALL = [
    dict(N=13, L=7.0, natoms=2, p=5, Z=5.0, seed=3),
    dict(N=11, L=6.0, natoms=3, p=70, Z=4.0, seed=4),
]


@pytest.fixture(params=SMALL, ids=["N13p5", "N11p70"])
def case(request):
    s = ki.small_system(**request.param)
    model = oe.Model.from_system(s)
    X = ost.m_orthonormalize(model, s.x0())
    return s, model, X


def test_vext_and_eii(case):
    s, model, X = case
    P = make(s)
    assert_rel(host(P.step_vext()), model.vext(), what="vext")
    assert P.step_eii() == pytest.approx(model.eii(), rel=1e-13)


def test_density(case):
    s, model, X = case
    P = make(s)
    assert_rel(host(P.step_density(dev(X))), oe.density(X, model.occ), what="rho")


@pytest.mark.parametrize("precond", [False, True], ids=["plain", "sine-preconditioned"])
def test_hartree_cg(case, precond):
    s, model, X = case
    P = make(s, cg_precond=precond)
    rho = oe.density(X, model.occ)
    b = 4 * math.pi * model.h ** 3 * rho
    v, r, it = P.step_hartree(dev(rho))
    v = host(v)
    # the oracle's own residual of the GPU potential meets the tolerance
    res = b - ofe.apply_K(v, model.N, model.h)
    assert np.linalg.norm(res) <= 1.05e-10 * np.linalg.norm(b)
    assert np.allclose(host(r), res, atol=1e-13 * np.abs(b).max())
    assert_rel(v, ofe.poisson_exact(b, model.N, model.h), rel=1e-8, what="vH vs exact")
    if precond:
        # the FP32 sine-basis inverse of K leaves only rounding-level error
        assert it <= 4
    else:
        # same iteration count as plain CG from the same start, same answer
        vo, ro, ito, ok = ofe.cg_solve(lambda x: ofe.apply_K(x, model.N, model.h), b, None,
                                       1e-10, 10000)
        assert ok and abs(it - ito) <= 1
        assert_rel(v, vo, rel=1e-9, what="vH vs oracle CG")
    # warm start from the answer converges immediately
    v2, _, it2 = P.step_hartree(dev(rho), dev(v), warm=True)
    assert it2 <= 1


@pytest.mark.parametrize("N", [140, 161])
def test_hartree_cg_tiled_preconditioner(N):
    # above N = 128 the sine-basis preconditioner runs as tiled axis passes
    # (ragged against the 64 x 128 tiles at both sizes): same answer and the
    # same two-to-four iterations as the fused form
    s = ki.config_of_al(cells=2)
    s.N, s.L = N, 0.4 * (N + 1)
    model = oe.Model.from_system(s)
    rng = np.random.default_rng(5)
    rho = rng.random(model.n)
    b = 4 * math.pi * model.h ** 3 * rho
    P = make(s)
    v, r, it = P.step_hartree(dev(rho))
    assert it <= 4
    v = host(v)
    res = b - ofe.apply_K(v, model.N, model.h)
    assert np.linalg.norm(res) <= 1.05e-10 * np.linalg.norm(b)
    assert_rel(v, ofe.poisson_exact(b, model.N, model.h), rel=1e-8, what="vH vs exact")


def test_potential_and_energies(case):
    s, model, X = case
    P = make(s)
    rho = oe.density(X, model.occ)
    b = 4 * math.pi * model.h ** 3 * rho
    vH = ofe.poisson_exact(b, model.N, model.h)
    rng = np.random.default_rng(1)
    resid = 1e-9 * rng.standard_normal(rho.shape)
    veff, e = P.step_potential(dev(rho), dev(vH), dev(resid))
    eps, vxc = oe.lda(rho, model.xc)
    h3 = model.h ** 3
    assert_rel(host(veff), model.vext() + vH + vxc, what="veff")
    assert e[0] == pytest.approx(h3 * model.vext() @ rho, rel=REL)
    assert e[1] == pytest.approx(0.5 * h3 * vH @ rho + vH @ resid / (8 * math.pi), rel=REL)
    assert e[2] == pytest.approx(h3 * rho @ eps, rel=REL)


def test_hamiltonian_stencil(case):
    s, model, X = case
    P = make(s)
    rng = np.random.default_rng(2)
    veff = rng.standard_normal(model.n)
    EX, MX, kin = P.step_hamiltonian(dev(X), dev(veff))
    KX = ofe.apply_K(X, model.N, model.h)
    want = model.occ * KX + 2 * model.occ * model.h ** 3 * veff[:, None] * X
    assert_rel(host(EX), want, what="E_X")
    assert_rel(host(MX), ofe.apply_M(X, model.N, model.h), what="MX")
    assert kin == pytest.approx(0.5 * model.occ * np.sum(X * KX), rel=REL)


def test_mass_and_inverse(case):
    s, model, X = case
    P = make(s)
    rng = np.random.default_rng(3)
    E = rng.standard_normal(X.shape)
    assert_rel(host(P.step_mass(dev(E))), ofe.apply_M(E, model.N, model.h), what="M E")
    assert_rel(host(P.step_mass_inverse(dev(E))), ofe.mass_inverse(E, model.N, model.h),
               rel=1e-11, what="M^-1 E")


def test_gram_and_combine(case):
    s, model, X = case
    P = make(s)
    rng = np.random.default_rng(4)
    A = rng.standard_normal(X.shape)
    B = rng.standard_normal(X.shape)
    assert_rel(host(P.step_gram(dev(A), dev(B))), A.T @ B, what="A^T B")
    C1 = rng.standard_normal((s.p, s.p))
    C2 = rng.standard_normal((s.p, s.p))
    out = P.step_combine(dev(A), dev(C1), dev(B), dev(C2), alpha=-0.5, beta=2.0, Bm=dev(X))
    assert_rel(host(out), -0.5 * (A @ C1 + B @ C2) + 2.0 * X, what="combine")


def test_energy_grad_and_projected_gradient(case):
    s, model, X = case
    P = make(s, cg_tol=1e-13)
    E, EX, D, g = P.energy_grad(dev(X), want_ex=True, want_d=True)
    ref = oe.evaluate(model, X)
    pt = ost.project(model, X, ref)
    assert E == pytest.approx(ref.E, rel=1e-12)
    assert_rel(host(EX), ref.EX, rel=1e-11, what="E_X")
    assert_rel(host(D), pt.D, rel=1e-10, what="D")
    assert g == pytest.approx(pt.dnorm, rel=1e-10)
    parts = P.energy_parts()
    for got, key in zip(parts, ["kinetic", "external", "hartree", "xc", "ion"]):
        assert got == pytest.approx(ref.parts[key], rel=1e-11, abs=1e-12)


@pytest.mark.parametrize("kind", ["qr", "cayley"])
def test_retract(case, kind):
    import paper_1308_2864_gb300 as ks
    s, model, X = case
    P = make(s)
    ref = oe.evaluate(model, X)
    pt = ost.project(model, X, ref)
    for tau in (1e-3, 0.05):
        got = host(P.retract(ks.KS_QR if kind == "qr" else ks.KS_CAYLEY, dev(X), dev(ref.EX), tau))
        want = (ost.retract_qr if kind == "qr" else ost.retract_cayley)(model, pt, tau)
        assert_rel(got, want, rel=1e-11, what=f"{kind} tau={tau}")
        assert ost.ortho_error(model, got) < 1e-12


def test_orthonormalize(case):
    s, model, X = case
    P = make(s)
    X0 = s.x0()
    got = host(P.orthonormalize(dev(X0)))
    assert_rel(got, ost.m_orthonormalize(model, X0), rel=1e-11, what="CholQR2")
    assert ost.ortho_error(model, got) < 1e-13


@pytest.mark.parametrize("retraction", ["qr", "cayley"])
def test_minimize_matches_oracle(retraction):
    # A case the oracle brute-force pins (resolved pseudo-atoms, rc = 1):
    # both sides converge to the same KKT point from the same start.
    s = ki.small_system(N=10, L=7.0, natoms=2, p=2, Z=1.0, seed=7)
    s.rc = 1.0
    model = oe.Model.from_system(s)
    ref = ost.minimize(model, s.x0(), ost.Options(retraction=retraction, gtol=1e-8, maxit=2000))
    assert ref.converged
    P = make(s)
    X = dev(s.x0())
    r = P.minimize(X, retraction=retraction, gtol=1e-8, maxit=2000)
    assert r["status"] == 0 and r["gradnorm"] <= 1e-8
    assert r["E"] == pytest.approx(ref.E, abs=1e-8)
    Xg = host(X)
    assert ost.ortho_error(model, Xg) < 1e-12
    # invariants: density and the Lagrange-multiplier spectrum
    assert_rel(oe.density(Xg, 2.0), oe.density(ref.X, 2.0), rel=1e-5, what="rho")
    lam_g = np.linalg.eigvalsh(Xg.T @ oe.evaluate(model, Xg).EX)
    lam_o = np.linalg.eigvalsh(ref.X.T @ ref.point.ev.EX)
    assert np.allclose(lam_g, lam_o, atol=1e-6)


def test_c1_trajectory_matches_oracle_early():
    # Config c1 (24^3, 2 atoms, p = 4, Slater, Cayley): the first 25
    # iterations follow the oracle's trajectory closely (BB steps amplify
    # rounding only slowly at the start).
    s = ki.config_c1()
    model = oe.Model.from_system(s)
    ref = ost.minimize(model, s.x0(), ost.Options(retraction="cayley", maxit=25))
    P = make(s)
    r = P.minimize(dev(s.x0()), retraction="cayley", maxit=25)
    assert r["iters"] == 25
    assert r["E"] == pytest.approx(ref.E, rel=1e-7)
    assert r["gradnorm"] == pytest.approx(ref.dnorm, rel=1e-4)


def test_host_entry_point_matches_device_entry_point():
    s = ki.small_system(N=9, L=6.0, natoms=1, p=3, Z=6.0, seed=2)
    P = make(s)
    Xh = np.ascontiguousarray(s.x0())
    rh = P.minimize_host(Xh, maxit=15)
    Xd = dev(s.x0())
    rd = P.minimize(Xd, maxit=15)
    assert rh["E"] == rd["E"]
    assert np.array_equal(Xh, host(Xd))


def test_invalid_arguments_are_reported():
    import paper_1308_2864_gb300 as ks
    with pytest.raises(ks.KSError) as e:
        ks.Problem(N=1, L=1.0, atoms=np.zeros((0, 3)), Z=np.zeros(0), p=1)
    assert e.value.status == ks.KS_EINVAL


def test_cg_limit_reports_noconv():
    import paper_1308_2864_gb300 as ks
    s = ki.small_system(N=12, L=6.0, natoms=1, p=2, Z=4.0, seed=1)
    P = make(s, cg_maxit=1, cg_precond=False)
    X = ost.m_orthonormalize(oe.Model.from_system(s), s.x0())
    with pytest.raises(ks.KSError) as e:
        P.step_hartree(P.step_density(dev(X)))
    assert e.value.status == ks.KS_ENOCONV


@pytest.mark.parametrize("retraction", ["qr", "cayley"])
def test_mixed_precision_then_fp64_polish(retraction):
    # FP32 orbital blocks down to ||D|| <= 1e-4, then the FP64 polish: the
    # final energy matches the FP64 oracle's minimiser like the FP64 run.
    s = ki.small_system(N=10, L=7.0, natoms=2, p=2, Z=1.0, seed=7)
    s.rc = 1.0
    model = oe.Model.from_system(s)
    ref = ost.minimize(model, s.x0(), ost.Options(retraction=retraction, gtol=1e-8, maxit=2000))
    P = make(s)
    X = dev(s.x0())
    r = P.minimize(X, retraction=retraction, gtol=1e-8, maxit=3000, precision="mixed",
                   polish_gtol=1e-4)
    assert r["status"] == 0 and r["gradnorm"] <= 1e-8
    assert r["mixed_iters"] > 0 and r["mixed_gradnorm"] <= 1e-3
    assert abs(r["mixed_E"] - ref.E) <= 1e-5
    assert r["E"] == pytest.approx(ref.E, abs=1e-8)
    assert ost.ortho_error(model, host(X)) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_checkpoint_resume_is_bitwise(precision):
    # 25 iterations + checkpoint + 20 more (in the same problem and after a
    # load into a fresh one) reproduce an uninterrupted 45-iteration run.
    s = ki.small_system(N=12, L=7.0, natoms=2, p=4, Z=4.0, seed=11)
    kw = dict(retraction="qr", gtol=1e-12, precision=precision, polish_gtol=1e-12,
              stall_iters=0)
    P = make(s)
    Xa = dev(s.x0())
    ra = P.minimize(Xa, maxit=45, **kw)
    P2 = make(s)
    Xb = dev(s.x0())
    P2.minimize(Xb, maxit=25, **kw)
    blob = P2.state_save()
    rb = P2.minimize(Xb, maxit=45, resume=1, **kw)
    P3 = make(s)
    P3.state_load(blob)
    Xc = torch.empty_like(Xb)
    rc = P3.minimize(Xc, maxit=45, resume=1, **kw)
    assert ra["E"] == rb["E"] == rc["E"]
    assert torch.equal(Xa, Xb) and torch.equal(Xa, Xc)
    assert rb["iters"] == 20 and rc["iters"] == 20


def test_failures_are_reported_and_leave_the_problem_usable():
    # host-visible failure paths on inputs that no kernel can fault on: a NaN
    # orbital entry (KS_ENAN from the energy and from the Hartree step) and a
    # zero column (KS_ENOTPD from the Cholesky factor, X left unchanged); the
    # same problem then evaluates a good block to the oracle's energy
    import paper_1308_2864_gb300 as ks
    s = ki.small_system(N=10, L=7.0, natoms=2, p=2, Z=2.0, seed=11)
    model = oe.Model.from_system(s)
    Xg = ost.m_orthonormalize(model, s.x0())
    ref = oe.evaluate(model, Xg).E
    P = make(s, cg_tol=1e-13)
    Xn = Xg.copy()
    Xn[123, 1] = float("nan")
    with pytest.raises(ks.KSError) as e:
        P.energy_grad(dev(Xn))
    assert e.value.status == ks.KS_ENAN
    rho = torch.full((s.n,), float("nan"), dtype=torch.float64, device="cuda")
    with pytest.raises(ks.KSError) as e:
        P.step_hartree(rho)
    assert e.value.status == ks.KS_ENAN
    Xz = Xg.copy()
    Xz[:, 1] = 0.0
    Xd = dev(Xz)
    with pytest.raises(ks.KSError) as e:
        P.orthonormalize(Xd)
    assert e.value.status == ks.KS_ENOTPD
    assert np.array_equal(host(Xd), Xz)
    E = P.energy_grad(dev(Xg))[0]
    assert E == pytest.approx(ref, rel=1e-11)
    Xo = P.orthonormalize(dev(s.x0()))
    assert ost.ortho_error(model, host(Xo)) < 1e-12


def test_workspace_calls_discard_the_saved_state():
    # ks_energy_grad, ks_retract and ks_orthonormalize reuse the blocks that
    # hold a minimisation's state, so afterwards there is nothing to resume
    import paper_1308_2864_gb300 as ks
    s = ki.small_system(N=10, L=7.0, natoms=2, p=2, Z=2.0, seed=11)
    kw = dict(retraction="qr", gtol=1e-12)
    for call in ("energy_grad", "retract", "orthonormalize"):
        P = make(s)
        X = dev(s.x0())
        P.minimize(X, maxit=5, **kw)
        assert len(P.state_save()) > 0
        if call == "energy_grad":
            P.energy_grad(X)
        elif call == "retract":
            E, EX, D, g = P.energy_grad(X, want_ex=True)
            P.minimize(X, maxit=5, **kw)
            P.retract(ks.KS_QR, X, EX, 1e-3)
        else:
            P.orthonormalize(X)
        with pytest.raises(ks.KSError):
            P.state_save()
        with pytest.raises(ks.KSError):
            P.minimize(X, maxit=10, resume=1, **kw)


def test_state_load_rejects_bad_checkpoints():
    # a checkpoint of another grid, a truncated one and one whose header
    # names an unknown retraction are refused; a refused load leaves nothing
    # to resume from, and the intact checkpoint still resumes
    import struct
    import paper_1308_2864_gb300 as ks
    s = ki.small_system(N=12, L=7.0, natoms=2, p=4, Z=4.0, seed=11)
    kw = dict(retraction="qr", gtol=1e-12)
    P = make(s)
    P.minimize(dev(s.x0()), maxit=5, **kw)
    blob = P.state_save()
    bad = bytearray(blob)
    struct.pack_into("<i", bad, 24, 7)           # u64 magic, i32 version, N, p, elem, retraction
    Q = make(s)
    for b in (bytes(bad), blob[:200], b"\0" * len(blob)):
        with pytest.raises(ks.KSError) as e:
            Q.state_load(b)
        assert e.value.status == ks.KS_EINVAL
    with pytest.raises(ks.KSError):
        Q.minimize(dev(s.x0()), maxit=10, resume=1, **kw)
    other = make(ki.small_system(N=11, L=7.0, natoms=2, p=4, Z=4.0, seed=11))
    with pytest.raises(ks.KSError):
        other.state_load(blob)
    Q.state_load(blob)
    r = Q.minimize(torch.empty((s.n, s.p), dtype=torch.float64, device="cuda"), maxit=10,
                   resume=1, **kw)
    assert r["iters"] == 5


@pytest.mark.parametrize("shape", [(13, 70, 70), (16, 64, 64), (11, 130, 70), (9, 12, 9),
                                   (9, 300, 260)])
@pytest.mark.parametrize("tc", [0, 2], ids=["fp32-pipes", "tensor-cores"])
def test_fp32_gram_tensor_cores(shape, tc):
    # FP32 Gram of the mixed phase: tensor cores (3 x TF32) for pa, qb > 8,
    # the register kernel below; compared with the exact FP64 product of
    # the same FP32 inputs.  n = N^3 rows is ragged against the 32-row stage.
    N, pa, qb = shape
    s = ki.small_system(N=N, L=7.0, natoms=2, p=max(pa, qb), Z=4.0, seed=4)
    P = make(s)
    P.set_tensor_cores(tc)
    rng = np.random.default_rng(21)
    A = rng.standard_normal((s.n, pa)).astype(np.float32)
    B = rng.standard_normal((s.n, qb)).astype(np.float32)
    got = host(P.step_gram_f32(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()))
    want = A.astype(np.float64).T @ B.astype(np.float64)
    # |A|^T |B| bounds the rounding of every entry
    bound = np.abs(A.astype(np.float64)).T @ np.abs(B.astype(np.float64))
    assert np.all(np.abs(got - want) <= 2e-6 * bound + 1e-12)


@pytest.mark.parametrize("shape", [(13, 70, 70), (16, 64, 64), (9, 40, 33), (11, 12, 20),
                                   (9, 300, 300), (12, 4, 8), (40, 64, 64)])
@pytest.mark.parametrize("tc", [0, 2, 3], ids=["fp32-pipes", "tensor-cores", "narrow-tc"])
def test_fp32_update_tensor_cores(shape, tc):
    # FP32 update X C1 + D C2 of the mixed phase (tensor cores for q > 32,
    # one thread per entry below; with tc = 3 the narrow form, q <= 64 and
    # widths a multiple of 4, takes the three terms as TMA stages of 128
    # rows, and a block accumulates its tiles in two alternating tensor-
    # memory accumulators: n = 40^3 gives 500 tiles, several per block),
    # against the exact FP64 result of the same FP32 inputs and the FP64 C
    # matrices.
    N, k, q = shape
    s = ki.small_system(N=N, L=7.0, natoms=2, p=max(k, q), Z=4.0, seed=4)
    P = make(s)
    P.set_tensor_cores(tc)
    rng = np.random.default_rng(23)
    A1 = rng.standard_normal((s.n, k)).astype(np.float32)
    A2 = rng.standard_normal((s.n, k)).astype(np.float32)
    Bm = rng.standard_normal((s.n, q)).astype(np.float32)
    C1 = rng.standard_normal((k, q))
    C2 = rng.standard_normal((k, q))
    t = lambda a: torch.from_numpy(a).cuda()
    got = host(P.step_combine_f32(t(A1), t(C1), t(A2), t(C2), alpha=-0.5, beta=2.0, Bm=t(Bm)))
    A1d, A2d = A1.astype(np.float64), A2.astype(np.float64)
    want = -0.5 * (A1d @ C1 + A2d @ C2) + 2.0 * Bm.astype(np.float64)
    bound = 0.5 * (np.abs(A1d) @ np.abs(C1) + np.abs(A2d) @ np.abs(C2)) + 2.0 * np.abs(Bm)
    assert np.all(np.abs(got - want) <= 4e-6 * bound + 1e-12)


# (N, p): p = 64 and 20 take the TMA ring in both precisions (row pitch a
# multiple of 16 bytes), p = 6 only in FP64, p = 5 in neither; N = 13 and 9
# leave ragged tiles in x, y and along z.
STAGING = [(13, 64), (9, 20), (13, 6), (9, 5)]


@pytest.mark.parametrize("shape", STAGING, ids=[f"N{n}p{p}" for n, p in STAGING])
def test_stencil_staging_paths_agree(shape):
    # TMA-staged and plain-load stencils form the same sums in the same
    # order: bitwise equal outputs in FP64 and FP32.
    N, p = shape
    s = ki.small_system(N=N, L=7.0, natoms=2, p=p, Z=4.0, seed=5)
    P = make(s)
    rng = np.random.default_rng(31)
    X = rng.standard_normal((s.n, p))
    veff = dev(rng.standard_normal(s.n))
    X64, X32 = dev(X), torch.from_numpy(X.astype(np.float32)).cuda()
    out = {}
    for mode in (0, 1):
        P.set_tma(mode)
        out[mode] = (P.step_hamiltonian(X64, veff), P.step_mass(X64),
                     P.step_hamiltonian_f32(X32, veff))
    (e0, m0, k0), mm0, (f0, fm0, fk0) = out[0]
    (e1, m1, k1), mm1, (f1, fm1, fk1) = out[1]
    assert torch.equal(e0, e1) and torch.equal(m0, m1) and torch.equal(mm0, mm1)
    assert torch.equal(f0, f1) and torch.equal(fm0, fm1)
    assert k0 == k1 and fk0 == fk1


@pytest.mark.parametrize("shape", [(13, 64), (9, 20), (11, 5)])
def test_fp32_hamiltonian_stencil(shape):
    # FP32 stencil of the mixed phase against the FP64 oracle on the same
    # FP32-rounded inputs: each entry sums 27 terms of FP32 products, so the
    # error is bounded by a few ulps of the sum of absolute terms.
    N, p = shape
    s = ki.small_system(N=N, L=7.0, natoms=2, p=p, Z=4.0, seed=6)
    model = oe.Model.from_system(s)
    P = make(s)
    rng = np.random.default_rng(32)
    X = rng.standard_normal((s.n, p)).astype(np.float32).astype(np.float64)
    veff = rng.standard_normal(s.n).astype(np.float32).astype(np.float64)
    EX, MX, kin = P.step_hamiltonian_f32(torch.from_numpy(X.astype(np.float32)).cuda(), dev(veff))
    KX = ofe.apply_K(X, model.N, model.h)
    want = model.occ * KX + 2 * model.occ * model.h ** 3 * veff[:, None] * X
    # sum of |terms|: |K| |X| is K with its off-centre entries negated, i.e.
    # 2 K0 |X| - K |X| with K0 the centre coefficient
    k0 = 2 * ofe.apply_K(np.eye(1, s.n, s.n // 2).T, model.N, model.h)[s.n // 2, 0]
    absKX = k0 * np.abs(X) - ofe.apply_K(np.abs(X), model.N, model.h)
    scale = (model.occ * absKX +
             2 * model.occ * model.h ** 3 * np.abs(veff)[:, None] * np.abs(X))
    err = np.abs(host(EX).astype(np.float64) - want)
    assert np.all(err <= 64 * 2.0 ** -24 * scale + 1e-30)
    mwant = ofe.apply_M(X, model.N, model.h)
    mscale = ofe.apply_M(np.abs(X), model.N, model.h)    # M is entrywise positive
    assert np.all(np.abs(host(MX).astype(np.float64) - mwant) <= 64 * 2.0 ** -24 * mscale)
    assert kin == pytest.approx(0.5 * model.occ * np.sum(X * KX), rel=1e-5)


def test_mixed_minimize_same_with_and_without_tma():
    # the whole mixed run (FP32 phase with every stencil kind, then the FP64
    # polish) is bitwise the same with either staging
    s = ki.small_system(N=12, L=7.0, natoms=2, p=8, Z=4.0, seed=12)
    kw = dict(retraction="qr", gtol=1e-7, maxit=60, precision="mixed", polish_gtol=1e-3)
    res, Xs = [], []
    for mode in (0, 1):
        P = make(s)
        P.set_tma(mode)
        X = dev(s.x0())
        res.append(P.minimize(X, **kw))
        Xs.append(X)
    assert res[0]["E"] == res[1]["E"] and res[0]["iters"] == res[1]["iters"]
    assert torch.equal(Xs[0], Xs[1])


@pytest.mark.parametrize("shape", [(9, 20, 13), (11, 32, 32), (8, 9, 31)])
def test_gram_mid_size(shape):
    # 8 < pa, qb <= 32: one thread per Gram entry, no padded tile
    N, pa, qb = shape
    s = ki.small_system(N=N, L=7.0, natoms=2, p=max(pa, qb), Z=4.0, seed=4)
    P = make(s)
    rng = np.random.default_rng(41)
    A = rng.standard_normal((s.n, pa))
    B = rng.standard_normal((s.n, qb))
    assert_rel(host(P.step_gram(dev(A), dev(B))), A.T @ B, rel=1e-13, what="A^T B")


def test_qr_retract_large_p():
    # p above the shared-memory limit of the p x p factor (global scratch)
    import paper_1308_2864_gb300 as ks
    s = ki.small_system(N=9, L=7.0, natoms=3, p=130, Z=4.0, seed=13)
    model = oe.Model.from_system(s)
    X = ost.m_orthonormalize(model, s.x0())
    P = make(s)
    ref = oe.evaluate(model, X)
    pt = ost.project(model, X, ref)
    for tau in (1e-3, 0.05):
        got = host(P.retract(ks.KS_QR, dev(X), dev(ref.EX), tau))
        assert_rel(got, ost.retract_qr(model, pt, tau), rel=1e-11, what=f"qr tau={tau}")
        assert ost.ortho_error(model, got) < 1e-12
    Y = dev(s.x0())
    P.orthonormalize(Y)
    assert ost.ortho_error(model, host(Y)) < 1e-12


@pytest.mark.parametrize("shape", [(13, 70, 70), (16, 64, 64), (11, 130, 70), (9, 12, 9),
                                   (45, 64, 64), (7, 1, 3)],
                         ids=["N13p70", "N16p64", "N11pa130qb70", "N9p12", "N45p64-chunks", "N7p1"])
def test_fp64_gram_on_tensor_cores(shape):
    # digit-split FP64 Grams (mode 2: always) against FP64 A^T B: every entry
    # within 2^-44 of sum_k |A_ki| |B_kj| (48 bits per operand below its
    # column maximum), on columns spanning 16 orders of magnitude, signs,
    # a zero column, and n beyond one 512-row chunk per block
    N, pa, qb = shape
    s = ki.small_system(N=N, L=7.0, natoms=2, p=max(pa, qb), seed=9)
    P = make(s)
    P.set_fp64_emulation(2)
    rng = np.random.default_rng(N * 1000 + pa)
    A = rng.standard_normal((N ** 3, pa)) * np.logspace(-8, 8, pa)[None, :]
    B = rng.standard_normal((N ** 3, qb)) * np.logspace(5, -5, qb)[None, :]
    if pa > 2:
        A[:, 1] = 0.0
    want = A.T @ B
    bound = np.abs(A).T @ np.abs(B)
    got = host(P.step_gram(dev(A), dev(B)))
    assert np.all(np.abs(got - want) <= 2.0 ** -44 * bound + 1e-300)
    P.set_fp64_emulation(0)
    ref = host(P.step_gram(dev(A), dev(B)))
    assert np.all(np.abs(ref - want) <= 1e-12 * bound + 1e-300)


@pytest.mark.parametrize("retraction", ["qr", "cayley"])
def test_fp64_emulated_grams_in_a_minimisation(retraction):
    s = ki.small_system(N=10, L=7.0, natoms=2, p=2, Z=1.0, seed=7)
    s.rc = 1.0
    model = oe.Model.from_system(s)
    ref = ost.minimize(model, s.x0(), ost.Options(retraction=retraction, gtol=1e-8, maxit=2000))
    P = make(s)
    P.set_fp64_emulation(2)
    X = dev(s.x0())
    r = P.minimize(X, retraction=retraction, gtol=1e-8, maxit=2000)
    assert r["status"] == 0 and r["gradnorm"] <= 1e-8
    assert r["E"] == pytest.approx(ref.E, abs=1e-8)
    assert ost.ortho_error(model, host(X)) < 1e-12


@pytest.mark.parametrize("shape", [(13, 64, 64, 64), (16, 32, 32, 70), (11, 5, 0, 5),
                                   (45, 64, 64, 64), (9, 100, 28, 50)],
                         ids=["N13k64+64q64", "N16k32+32q70", "N11k5q5", "N45k64+64q64",
                              "N9k100+28q50"])
def test_fp64_update_on_tensor_cores(shape):
    # digit-split FP64 update out = alpha (A1 C1 + A2 C2) + beta Bm against
    # FP64.  Each row of [A1 A2] and each column of [C1; C2] is split into 56
    # bits below its own largest entry, so an entry of the product is within
    # K 2^-50 max_k |A_ik| max_k |C_kj| (truncation and the dropped digit
    # pairs) plus the FP64 rounding of the result; rows and columns span 12
    # orders of magnitude
    N, k1, k2, q = shape
    s = ki.small_system(N=N, L=7.0, natoms=2, p=max(k1, k2, q), seed=9)
    P = make(s)
    P.set_fp64_emulation(2)
    rng = np.random.default_rng(N * 100 + k1 + q)
    n = N ** 3
    A1 = rng.standard_normal((n, k1)) * np.logspace(-6, 6, n)[:, None]
    C1 = rng.standard_normal((k1, q)) * np.logspace(3, -3, q)[None, :]
    A2 = rng.standard_normal((n, k2)) if k2 else None
    C2 = rng.standard_normal((k2, q)) if k2 else None
    Bm = rng.standard_normal((n, q))
    alpha, beta = -0.75, 1.5
    A = np.hstack([A1, A2]) if k2 else A1
    C = np.vstack([C1, C2]) if k2 else C1
    prod = A @ C
    split = (k1 + k2) * 2.0 ** -50 * np.abs(A).max(axis=1)[:, None] * np.abs(C).max(axis=0)[None, :]
    got = host(P.step_combine(dev(A1), dev(C1), dev(A2) if k2 else None,
                              dev(C2) if k2 else None, alpha=alpha, beta=beta, Bm=dev(Bm)))
    want = alpha * prod + beta * Bm
    tol = abs(alpha) * split + 4 * 2.0 ** -53 * (np.abs(alpha * prod) + np.abs(beta * Bm))
    assert np.all(np.abs(got - want) <= tol)
    got0 = host(P.step_combine(dev(A1), dev(C1), dev(A2) if k2 else None,
                               dev(C2) if k2 else None, alpha=1.0, beta=0.0))
    assert np.all(np.abs(got0 - prod) <= split + 4 * 2.0 ** -53 * np.abs(prod))


def test_fp64_split_products_reach_the_same_minimiser():
    # 48 orbitals (the split applies to Grams with >= 48 columns and to the
    # updates): plain FP64 and split products converge to the same energy
    import paper_1308_2864_gb300 as ks
    s = ki.small_system(N=14, L=8.0, natoms=24, p=48, Z=4.0, seed=5)
    s.rc = 1.0
    E = []
    for mode in (0, 1):
        P = make(s)
        P.set_fp64_emulation(mode)
        X = dev(s.x0())
        r = P.minimize(X, gtol=1e-6, maxit=20000)
        assert r["status"] == 0 and r["gradnorm"] <= 1e-6
        E.append(r["E"])
        assert ost.ortho_error(oe.Model.from_system(s), host(X)) < 1e-11
    assert E[1] == pytest.approx(E[0], abs=1e-9)


def test_bounded_wait_expires_and_the_context_survives():
    # a grid-barrier wait that nothing completes gives up after its spin
    # limit and records KS_ETIMEOUT; the next launches run normally
    import paper_1308_2864_gb300 as ks
    st, sec = ks.selftest_wait_timeout()
    assert st == ks.KS_ETIMEOUT
    assert sec < 60.0
    s = ki.small_system(N=10, L=7.0, natoms=2, p=2, Z=2.0, seed=11)
    model = oe.Model.from_system(s)
    Xg = ost.m_orthonormalize(model, s.x0())
    E = make(s, cg_tol=1e-13).energy_grad(dev(Xg))[0]
    assert E == pytest.approx(oe.evaluate(model, Xg).E, rel=1e-11)
