"""Host-side argument checks of the C ABI, run without a GPU: every rejected
call returns KS_EINVAL with its reason before any device call, the option
defaults match the values include/ks.h documents, and a valid problem
without a device fails with a CUDA error instead of falling back to the CPU."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import paper_1308_2864_gb300 as ks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return ks.load_library()


def valid_desc(**kw):
    """Two hydrogen-like atoms on a 9^3 grid; keyword overrides per field."""
    atoms = np.array([[2.0, 2.0, 2.0], [3.0, 3.0, 3.0]])
    Z = np.array([1.0, 1.0])
    d = ks.ProblemDesc()
    d.N, d.L, d.natoms = 9, 5.0, 2
    d.R = atoms.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.Z = Z.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.rc, d.p, d.occ, d.xc = 0.5, 2, 2.0, ks.KS_XC_SLATER_PZ81
    d.cg_tol, d.cg_maxit, d.precision, d.cg_precond = 1e-10, 100, ks.KS_FP64, 1
    d.kinetic, d.mu, d.mass = ks.KS_KIN_ORBITALS, 1.0, ks.KS_MASS_CONSISTENT
    for k, v in kw.items():
        setattr(d, k, v)
    return d, (atoms, Z)


NULL_R = ctypes.POINTER(ctypes.c_double)()

# (field overrides, a word the recorded reason contains)
BAD_DESCS = [
    ({"N": 1}, "N = 1"), ({"N": 2049}, "N = 2049"),
    ({"L": 0.0}, "L must"), ({"L": -1.0}, "L must"), ({"L": math.nan}, "L must"),
    ({"p": 0}, "p = 0"), ({"N": 2, "p": 9}, "p = 9"),
    ({"N": 1291, "p": 1}, "2^31"), ({"N": 2048, "p": 1}, "2^31"), ({"N": 128, "p": 1024}, "2^31"),
    ({"natoms": -1}, "atom"), ({"R": NULL_R}, "atom"), ({"Z": NULL_R}, "atom"),
    ({"rc": 0.0}, "rc"), ({"xc": 7}, "xc"), ({"precision": 2}, "precision"),
    ({"cg_tol": 0.0}, "CG"), ({"cg_maxit": 0}, "CG"),
    ({"mass": 2}, "mass"), ({"kinetic": 2}, "kinetic"),
    ({"kinetic": ks.KS_KIN_TFW}, "p = 1"),
    ({"kinetic": ks.KS_KIN_TFW, "p": 1, "mu": -0.5}, "mu"),
    ({"kinetic": ks.KS_KIN_TFW, "p": 1, "mu": math.inf}, "mu"),
    ({"kinetic": ks.KS_KIN_TFW, "p": 1, "mu": math.nan}, "mu"),
]


def last_error(lib) -> str:
    return lib.ks_last_error_string().decode()


@pytest.mark.parametrize("bad,why", BAD_DESCS)
def test_problem_create_rejects_bad_descriptions(lib, bad, why):
    d, keep = valid_desc(**bad)
    h = ctypes.c_void_p(12345)
    assert lib.ks_problem_create(ctypes.byref(d), ctypes.byref(h)) == ks.KS_EINVAL
    assert h.value is None                      # *out cleared on failure
    assert why in last_error(lib)
    assert lib.ks_problem_bytes(ctypes.byref(d)) == 0


def test_problem_create_rejects_null_arguments(lib):
    d, keep = valid_desc()
    assert lib.ks_problem_create(ctypes.byref(d), None) == ks.KS_EINVAL
    h = ctypes.c_void_p()
    assert lib.ks_problem_create(None, ctypes.byref(h)) == ks.KS_EINVAL
    assert lib.ks_problem_bytes(None) == 0


def test_problem_bytes_of_valid_descriptions(lib):
    # the admission size grows with the grid and with the orbital count
    sizes = {}
    for N, p in [(9, 2), (17, 2), (17, 8)]:
        d, keep = valid_desc(N=N, p=p)
        sizes[N, p] = lib.ks_problem_bytes(ctypes.byref(d))
    assert 0 < sizes[9, 2] < sizes[17, 2] < sizes[17, 8]
    # at least the orbital-sized blocks: X, E_X, M X, D and the trial blocks
    assert sizes[17, 8] > 5 * 17 ** 3 * 8 * 8
    d, keep = valid_desc(kinetic=ks.KS_KIN_TFW, p=1, mu=0.0, mass=ks.KS_MASS_LUMPED)
    assert lib.ks_problem_bytes(ctypes.byref(d)) > 0
    # the largest grids with 32-bit entry indices: sizes computed without overflow
    for N, p in [(1290, 1), (128, 1023)]:
        d, keep = valid_desc(N=N, p=p)
        assert lib.ks_problem_bytes(ctypes.byref(d)) > 13 * N ** 3 * p * 8


def test_valid_problem_without_a_device_is_a_cuda_error(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    d, keep = valid_desc()
    h = ctypes.c_void_p()
    assert lib.ks_problem_create(ctypes.byref(d), ctypes.byref(h)) == ks.KS_ECUDA
    assert h.value is None


def test_batch_create_checks_every_description_first(lib):
    good, k1 = valid_desc()
    cases = [
        (valid_desc(p=105, N=9), "p > 104"),
        (valid_desc(kinetic=ks.KS_KIN_TFW, p=1), "orbital-free"),
        (valid_desc(mass=ks.KS_MASS_LUMPED), "lumped"),
        (valid_desc(N=1), "N = 1"),
    ]
    for (bad, k2), why in cases:
        arr = (ks.ProblemDesc * 2)(good, bad)
        h = ctypes.c_void_p(7)
        assert lib.ks_batch_create(arr, 2, None, ctypes.byref(h)) == ks.KS_EINVAL
        assert h.value is None
        assert why in last_error(lib), (why, last_error(lib))
    arr = (ks.ProblemDesc * 1)(good)
    h = ctypes.c_void_p()
    assert lib.ks_batch_create(arr, 0, None, ctypes.byref(h)) == ks.KS_EINVAL
    assert lib.ks_batch_create(None, 1, None, ctypes.byref(h)) == ks.KS_EINVAL


def test_minimize_refine_checks_before_device_calls(lib):
    o = ks.Opts()
    lib.ks_opts_default(ctypes.byref(o))
    res = (ks.Result * 4)()
    x0 = np.zeros(1000)
    xp = x0.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def call(d, levels, gtol=1e-3, x=xp, r=res):
        return lib.ks_minimize_refine(ctypes.byref(d), levels, x, ctypes.byref(o), gtol, None, r)

    d15, k = valid_desc(N=15)
    assert call(d15, 0) == ks.KS_EINVAL
    assert call(d15, 11) == ks.KS_EINVAL
    d12, k = valid_desc(N=12)
    assert call(d12, 2) == ks.KS_EINVAL and "divisible" in last_error(lib)
    d7, k = valid_desc(N=7)
    assert call(d7, 3) == ks.KS_EINVAL and "coarsest" in last_error(lib)   # 8 / 4 - 1 = 1
    assert call(d15, 2, gtol=0.0) == ks.KS_EINVAL and "coarse_gtol" in last_error(lib)
    assert call(d15, 2, gtol=math.nan) == ks.KS_EINVAL
    assert call(d15, 2, x=None) == ks.KS_EINVAL
    assert call(d15, 2, r=None) == ks.KS_EINVAL
    bad, k = valid_desc(N=15, kinetic=5)
    assert call(bad, 2) == ks.KS_EINVAL and "kinetic" in last_error(lib)


def test_prolong_checks_before_device_calls(lib):
    # addresses only compared, never dereferenced: every call here is rejected
    a, b = 1 << 20, 1 << 24
    for f in (lib.ks_prolong, lib.ks_prolong_f32):
        assert f(0, 1, a, b, None) == ks.KS_EINVAL
        assert f(1024, 1, a, b, None) == ks.KS_EINVAL
        assert f(2, 0, a, b, None) == ks.KS_EINVAL
        assert f(2, 1, None, b, None) == ks.KS_EINVAL
        assert f(2, 1, a, None, None) == ks.KS_EINVAL
        assert f(2, 1, a, a + 8, None) == ks.KS_EINVAL and "overlap" in last_error(lib)
        assert f(2, 1, a + 8, a, None) == ks.KS_EINVAL   # fine block (125 entries) covers a + 8
    # Nc = 2, p = 1: 8 coarse entries at a, 125 fine ones ending one entry
    # past a, so the last fine entry is the first coarse one
    assert lib.ks_prolong(2, 1, a, a - 124 * 8, None) == ks.KS_EINVAL


def test_null_handles_are_rejected(lib):
    o = ks.Opts()
    lib.ks_opts_default(ctypes.byref(o))
    r = ks.Result()
    e = ctypes.c_double()
    buf = ctypes.create_string_buffer(64)
    x = 1 << 20
    assert lib.ks_minimize(None, x, ctypes.byref(o), ctypes.byref(r)) == ks.KS_EINVAL
    assert lib.ks_minimize_host(None, None, ctypes.byref(o), ctypes.byref(r)) == ks.KS_EINVAL
    assert lib.ks_energy_grad(None, x, ctypes.byref(e), x, x, None) == ks.KS_EINVAL
    assert lib.ks_retract(None, ks.KS_QR, x, x, 1e-3, x) == ks.KS_EINVAL
    assert lib.ks_orthonormalize(None, x) == ks.KS_EINVAL
    assert lib.ks_state_save(None, buf, 64) == ks.KS_EINVAL
    assert lib.ks_state_load(None, buf, 64) == ks.KS_EINVAL
    for f in (lib.ks_set_tensor_cores, lib.ks_set_tma, lib.ks_set_fp64_emulation):
        assert f(None, 1) == ks.KS_EINVAL
    assert lib.ks_step_gram(None, x, 1, x, 1, x) == ks.KS_EINVAL
    assert lib.ks_step_mass_inverse(None, x, x) == ks.KS_EINVAL
    assert lib.ks_batch_set_graphs(None, 1) == ks.KS_EINVAL
    out = (ctypes.c_int * 4)()
    assert lib.ks_batch_autotune(None, out) == ks.KS_EINVAL
    assert lib.ks_batch_minimize(None, None, ctypes.byref(o), None) == ks.KS_EINVAL
    h = ctypes.c_void_p()
    assert lib.ks_server_create(1 << 30, 0, ctypes.byref(h)) == ks.KS_EINVAL
    assert lib.ks_server_create(1 << 30, 257, ctypes.byref(h)) == ks.KS_EINVAL
    assert lib.ks_server_create(0, 4, ctypes.byref(h)) == ks.KS_EINVAL
    assert lib.ks_server_create(1 << 30, 4, None) == ks.KS_EINVAL
    assert lib.ks_selftest_wait_timeout(None, None, None) == ks.KS_EINVAL


def documented_defaults() -> dict:
    """{field: value} from the ks_opts comments in include/ks.h: the last
    parenthesised number or KS_ constant of each field's comment."""
    txt = open(os.path.join(ROOT, "include", "ks.h")).read()
    body = txt[txt.index("typedef struct {", txt.index("Parameters of Alg. ConOptM")):]
    body = body[:body.index("} ks_opts;")]
    consts = {"KS_QR": ks.KS_QR, "KS_CAYLEY": ks.KS_CAYLEY, "KS_FP64": ks.KS_FP64,
              "KS_MIXED": ks.KS_MIXED}
    out = {}
    for m in re.finditer(r"(?:int|double)\s+(\w+);\s*/\*(.*?)\*/", body, re.S):
        vals = []
        for g in re.findall(r"\(([^()]*)\)", m.group(2)):
            g = g.strip()
            if g in consts:
                vals.append(consts[g])
            else:
                try:
                    vals.append(float(g))
                except ValueError:
                    pass
        assert vals, f"no documented default for {m.group(1)}"
        out[m.group(1)] = vals[-1]
    return out


def test_option_defaults_match_the_header(lib):
    doc = documented_defaults()
    assert set(doc) == {f for f, _ in ks.Opts._fields_}
    o = ks.Opts()
    lib.ks_opts_default(ctypes.byref(o))
    for f, v in doc.items():
        assert getattr(o, f) == v, (f, getattr(o, f), v)
    # the binding's defaults are the library's
    b = ks.default_opts()
    for f, _ in ks.Opts._fields_:
        assert getattr(b, f) == getattr(o, f), f


def test_binding_batch_refuses_unsupported_jobs_before_device_calls():
    # the Python job table marshals each system through the same description
    # as the single-system path; refused jobs raise before any device work
    import ks_inputs as ki
    ok = ki.small_system(N=8, L=6.0, natoms=1, p=2, Z=4.0, seed=3)
    for bad, why in [(ki.small_of_system(N=8), "orbital-free"),
                     (ki.small_system(N=8, L=6.0, natoms=1, p=105, Z=4.0, seed=3), "p > 104")]:
        with pytest.raises(ks.KSError) as e:
            ks.Batch([ok, bad])
        assert e.value.status == ks.KS_EINVAL and why in str(e.value)
