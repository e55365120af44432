"""The allocation-free Gram entry point (ks_gram_noalloc), called through the
C ABI, against the problem-based entry point (ks_step_gram).  It exists for
callers that cannot allocate device memory: processes whose device memory is
owned by their own allocator or reserved under a fixed budget, and code that
must not call into the CUDA allocator.  Its scratch is a file-scope device
array instead of memory from cudaMalloc.  Kept in a file of its own that
pytest collects last."""
import ctypes

import numpy as np
import pytest

import ks_inputs as ki

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(got, want):
    return float((got - want).abs().max() / want.abs().max())


def test_noalloc_gram_matches_problem_gram_twice():
    import paper_1308_2864_gb300 as ks
    lib = ks.load_library()
    # ragged sizes: n = 13^3 rows, p = 70 columns (two 64-wide tiles)
    s = ki.small_system(N=13, L=7.0, natoms=2, p=70, Z=4.0, seed=3)
    P = ks.Problem.from_system(s)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(17)
    for _ in range(2):
        A = torch.from_numpy(rng.standard_normal((s.n, s.p))).cuda()
        B = torch.from_numpy(rng.standard_normal((s.n, s.p - 3))).cuda()
        want = P.step_gram(A, B)
        out = torch.full((s.p, s.p - 3), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.ks_gram_noalloc(A.data_ptr(), s.p, B.data_ptr(), s.p - 3, s.n, out.data_ptr(),
                                 ctypes.c_void_p(stream.cuda_stream))
        assert st == ks.KS_OK
        stream.synchronize()
        assert _rel(out, want) <= 1e-12


def test_noalloc_gram_small_widths_twice():
    # widths below one 64-wide tile (the padded tile path), two calls in a row
    import paper_1308_2864_gb300 as ks
    lib = ks.load_library()
    s = ki.small_system(N=11, L=6.0, natoms=1, p=8, Z=2.0, seed=9)
    P = ks.Problem.from_system(s)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(23)
    for pa, qb in ((5, 3), (1, 8)):
        A = torch.from_numpy(rng.standard_normal((s.n, pa))).cuda()
        B = torch.from_numpy(rng.standard_normal((s.n, qb))).cuda()
        want = P.step_gram(A, B)
        out = torch.full((pa, qb), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.ks_gram_noalloc(A.data_ptr(), pa, B.data_ptr(), qb, s.n, out.data_ptr(),
                                 ctypes.c_void_p(stream.cuda_stream))
        assert st == ks.KS_OK
        stream.synchronize()
        assert _rel(out, want) <= 1e-12


def test_noalloc_gram_rejects_sizes_beyond_its_scratch():
    import paper_1308_2864_gb300 as ks
    lib = ks.load_library()
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = lib.ks_gram_noalloc(dummy.data_ptr(), 4096, dummy.data_ptr(), 4096, 1, dummy.data_ptr(),
                             None)
    assert st == ks.KS_EINVAL
    assert b"scratch" in lib.ks_last_error_string()
