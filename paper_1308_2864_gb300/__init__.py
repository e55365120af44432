"""Python binding of the GB300 Kohn-Sham minimisation library (C ABI in
include/ks.h and include/ks_steps.h).

This module only marshals arguments: device buffers are torch tensors on the
current CUDA device (FP64, contiguous, row-major n x p with the orbital index
fastest) whose data pointers are handed to the library, and all arithmetic
runs in the library's CUDA kernels.  There is no CPU fallback: importing
works without a GPU, but every call needs the compiled library and a CUDA
device, and raises otherwise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

(KS_OK, KS_EINVAL, KS_ENOMEM, KS_ECUDA, KS_ENOCONV, KS_ENOTPD, KS_ESINGULAR, KS_ENAN, KS_ETIMEOUT,
 KS_EAGAIN) = range(10)
STATUS_NAMES = ["KS_OK", "KS_EINVAL", "KS_ENOMEM", "KS_ECUDA", "KS_ENOCONV", "KS_ENOTPD",
                "KS_ESINGULAR", "KS_ENAN", "KS_ETIMEOUT", "KS_EAGAIN"]
KS_XC_SLATER, KS_XC_SLATER_PZ81 = 0, 1
KS_FP64, KS_MIXED = 0, 1
KS_QR, KS_CAYLEY = 0, 1
KS_KIN_ORBITALS, KS_KIN_TFW = 0, 1
KS_MASS_CONSISTENT, KS_MASS_LUMPED = 0, 1


class KSError(RuntimeError):
    def __init__(self, status: int, message: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")
        self.status = status


class ProblemDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("L", ctypes.c_double), ("natoms", ctypes.c_int),
                ("R", ctypes.POINTER(ctypes.c_double)), ("Z", ctypes.POINTER(ctypes.c_double)),
                ("rc", ctypes.c_double), ("p", ctypes.c_int), ("occ", ctypes.c_double),
                ("xc", ctypes.c_int), ("cg_tol", ctypes.c_double), ("cg_maxit", ctypes.c_int),
                ("precision", ctypes.c_int), ("stream", ctypes.c_void_p), ("cg_precond", ctypes.c_int),
                ("kinetic", ctypes.c_int), ("mu", ctypes.c_double), ("mass", ctypes.c_int)]


class Opts(ctypes.Structure):
    _fields_ = [("retraction", ctypes.c_int), ("gtol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("tau0", ctypes.c_double), ("rho1", ctypes.c_double), ("delta", ctypes.c_double),
                ("eta", ctypes.c_double), ("tau_min", ctypes.c_double), ("tau_max", ctypes.c_double),
                ("max_backtrack", ctypes.c_int), ("ortho_tol", ctypes.c_double),
                ("ortho_every", ctypes.c_int), ("verbose", ctypes.c_int),
                ("precision", ctypes.c_int), ("polish_gtol", ctypes.c_double),
                ("stall_iters", ctypes.c_int), ("stall_df", ctypes.c_double),
                ("resume", ctypes.c_int), ("mixed_cg_tol", ctypes.c_double),
                ("fp64_split", ctypes.c_int), ("fp32_increment", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("gradnorm", ctypes.c_double), ("ortho_err", ctypes.c_double),
                ("E_parts", ctypes.c_double * 5), ("iters", ctypes.c_int),
                ("cg_iters_total", ctypes.c_int), ("backtracks", ctypes.c_int),
                ("status", ctypes.c_int), ("seconds", ctypes.c_double),
                ("mixed_iters", ctypes.c_int), ("mixed_gradnorm", ctypes.c_double),
                ("mixed_E", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int), ("running", ctypes.c_int), ("peak_running", ctypes.c_int),
                ("completed", ctypes.c_ulonglong), ("bytes_in_use", ctypes.c_size_t),
                ("peak_bytes_in_use", ctypes.c_size_t), ("budget", ctypes.c_size_t)]


_LIB = None
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_DP = ctypes.POINTER(ctypes.c_double)

# (name, restype, argtypes) of every exported function.
SIGNATURES = [
    ("ks_opts_default", None, [ctypes.POINTER(Opts)]),
    ("ks_problem_create", _I, [ctypes.POINTER(ProblemDesc), ctypes.POINTER(_P)]),
    ("ks_problem_destroy", _I, [_P]),
    ("ks_problem_bytes", ctypes.c_size_t, [ctypes.POINTER(ProblemDesc)]),
    ("ks_energy_grad", _I, [_P, _P, _DP, _P, _P, _DP]),
    ("ks_energy_parts", _I, [_P, _DP]),
    ("ks_retract", _I, [_P, _I, _P, _P, _D, _P]),
    ("ks_orthonormalize", _I, [_P, _P]),
    ("ks_minimize", _I, [_P, _P, ctypes.POINTER(Opts), ctypes.POINTER(Result)]),
    ("ks_minimize_host", _I, [_P, _DP, ctypes.POINTER(Opts), ctypes.POINTER(Result)]),
    ("ks_prolong", _I, [_I, _I, _P, _P, _P]),
    ("ks_prolong_f32", _I, [_I, _I, _P, _P, _P]),
    ("ks_minimize_refine", _I, [ctypes.POINTER(ProblemDesc), _I, _DP, ctypes.POINTER(Opts), _D,
                                _DP, ctypes.POINTER(Result)]),
    ("ks_last_error_string", ctypes.c_char_p, []),
    ("ks_kernel_launches", ctypes.c_ulonglong, []),
    ("ks_debug_bounds", ctypes.c_int, [ctypes.POINTER(ctypes.c_ulonglong),
                                        ctypes.POINTER(ctypes.c_char_p),
                                        ctypes.POINTER(ctypes.c_int)]),
    ("ks_state_bytes", ctypes.c_size_t, [_P]),
    ("ks_state_save", _I, [_P, ctypes.c_void_p, ctypes.c_size_t]),
    ("ks_state_load", _I, [_P, ctypes.c_void_p, ctypes.c_size_t]),
    ("ks_profile_start", _I, []),
    ("ks_profile_stop", _I, [_DP, ctypes.POINTER(ctypes.c_longlong)]),
    ("ks_profile_class_name", ctypes.c_char_p, [_I]),
    ("ks_profile_work", _I, [_DP, _DP]),
    ("ks_step_vext", _I, [_P, _P]),
    ("ks_step_eii", _I, [_P, _DP]),
    ("ks_step_density", _I, [_P, _P, _P]),
    ("ks_step_hartree", _I, [_P, _P, _P, _I, _P, ctypes.POINTER(_I)]),
    ("ks_step_potential", _I, [_P, _P, _P, _P, _P, _DP]),
    ("ks_step_hamiltonian", _I, [_P, _P, _P, _P, _P, _DP]),
    ("ks_step_hamiltonian_f32", _I, [_P, _P, _P, _P, _P, _DP]),
    ("ks_step_mass", _I, [_P, _P, _P]),
    ("ks_step_mass_inverse", _I, [_P, _P, _P]),
    ("ks_step_gram", _I, [_P, _P, _I, _P, _I, _P]),
    ("ks_step_gram_f32", _I, [_P, _P, _I, _P, _I, _P]),
    ("ks_set_tensor_cores", _I, [_P, _I]),
    ("ks_set_tma", _I, [_P, _I]),
    ("ks_set_fp64_emulation", _I, [_P, _I]),
    ("ks_step_combine_f32", _I, [_P, _P, _I, _P, _P, _I, _P, _D, _D, _P, _P, _I]),
    ("ks_step_combine", _I, [_P, _P, _I, _P, _P, _I, _P, _D, _D, _P, _P, _I]),
    ("ks_gram_noalloc", _I, [_P, _I, _P, _I, ctypes.c_longlong, _P, _P]),
    ("ks_selftest_wait_timeout", _I, [_P, ctypes.POINTER(_I), _DP]),
    ("ks_probe_fma", _I, [_I, _I, _I, _P, _P, _DP]),
    ("ks_server_create", _I, [ctypes.c_size_t, _I, ctypes.POINTER(_P)]),
    ("ks_server_submit", _I, [_P, ctypes.POINTER(ProblemDesc), ctypes.POINTER(Opts), _DP,
                              ctypes.POINTER(ctypes.c_uint64)]),
    ("ks_server_poll", _I, [_P, ctypes.c_uint64, _I, ctypes.POINTER(Result), _DP, _DP]),
    ("ks_server_stats", _I, [_P, ctypes.POINTER(ServerStats)]),
    ("ks_server_destroy", _I, [_P]),
    ("ks_batch_create", _I, [ctypes.POINTER(ProblemDesc), _I, _P, ctypes.POINTER(_P)]),
    ("ks_batch_bytes", ctypes.c_size_t, [_P]),
    ("ks_batch_set_graphs", _I, [_P, _I]),
    ("ks_batch_autotune", _I, [_P, ctypes.POINTER(_I)]),
    ("ks_batch_minimize", _I, [_P, ctypes.POINTER(_DP), ctypes.POINTER(Opts),
                               ctypes.POINTER(Result)]),
    ("ks_batch_destroy", _I, [_P]),
]


def library_path() -> str:
    return _build.lib_path()


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load the compiled library (building it first when missing or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if build_if_missing and (_build.needs_build()):
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not found at {path}; run build() first")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(status: int):
    if status != KS_OK:
        msg = load_library().ks_last_error_string()
        raise KSError(status, msg.decode() if msg else "")


def _ptr32(t) -> int | None:
    """Device pointer of a CUDA FP32 contiguous tensor (None passes NULL)."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("expected a contiguous torch.float32 CUDA tensor")
    return t.data_ptr()


def _ptr(t) -> int | None:
    """Device pointer of a CUDA FP64 contiguous tensor (None passes NULL)."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous torch.float64 CUDA tensor")
    return t.data_ptr()


def default_opts(**kw) -> Opts:
    o = Opts()
    load_library().ks_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "retraction" and isinstance(v, str):
            v = KS_QR if v == "qr" else KS_CAYLEY
        if k == "precision" and isinstance(v, str):
            v = KS_FP64 if v == "fp64" else KS_MIXED
        if not hasattr(o, k):
            raise KeyError(f"unknown option {k}")
        setattr(o, k, v)
    return o


PROF_CLASSES = 12


def kernel_launches() -> int:
    """Kernels the library has launched in this process."""
    return int(load_library().ks_kernel_launches())


def debug_bounds() -> dict:
    """The bounds-checked build's record (ks_debug_bounds): whether the library
    is such a build, the out-of-range indices caught since the last call and
    where the first one was; the record is cleared."""
    c = ctypes.c_ulonglong()
    f = ctypes.c_char_p()
    ln = ctypes.c_int()
    checked = load_library().ks_debug_bounds(ctypes.byref(c), ctypes.byref(f), ctypes.byref(ln))
    return {"checked": bool(checked), "count": int(c.value),
            "file": f.value.decode() if f.value else None, "line": int(ln.value)}


def profile_start():
    _check(load_library().ks_profile_start())


def profile_stop() -> dict:
    """{class name: (milliseconds, timed launch groups, flops, DRAM bytes)}
    since profile_start() (algorithmic work, see ks_profile_work)."""
    lib = load_library()
    ms = (ctypes.c_double * PROF_CLASSES)()
    cnt = (ctypes.c_longlong * PROF_CLASSES)()
    fl = (ctypes.c_double * PROF_CLASSES)()
    by = (ctypes.c_double * PROF_CLASSES)()
    _check(lib.ks_profile_stop(ms, cnt))
    _check(lib.ks_profile_work(fl, by))
    return {lib.ks_profile_class_name(i).decode(): (ms[i], cnt[i], fl[i], by[i])
            for i in range(PROF_CLASSES)}


def result_dict(r: Result) -> dict:
    return {"E": r.E, "gradnorm": r.gradnorm, "ortho_err": r.ortho_err,
            "E_parts": list(r.E_parts), "iters": r.iters, "cg_iters_total": r.cg_iters_total,
            "backtracks": r.backtracks, "status": r.status, "seconds": r.seconds,
            "mixed_iters": r.mixed_iters, "mixed_gradnorm": r.mixed_gradnorm, "mixed_E": r.mixed_E}


def _system_desc(s, N: int | None = None, stream=None):
    """ProblemDesc of a ks_inputs.System (and the arrays it points into)."""
    atoms = np.ascontiguousarray(np.asarray(s.atoms, dtype=np.float64).reshape(-1, 3))
    Z = np.ascontiguousarray(np.asarray(s.Z, dtype=np.float64).reshape(-1))
    d = ProblemDesc()
    d.N, d.L, d.natoms = s.N if N is None else N, s.L, len(Z)
    d.R = atoms.ctypes.data_as(_DP)
    d.Z = Z.ctypes.data_as(_DP)
    d.rc, d.p, d.occ, d.xc = s.rc, s.p, s.occ, s.xc
    d.cg_tol, d.cg_maxit, d.precision, d.cg_precond = 1e-10, 20000, KS_FP64, 1
    d.kinetic, d.mu = getattr(s, "kinetic", KS_KIN_ORBITALS), getattr(s, "mu", 1.0)
    d.mass = getattr(s, "mass", KS_MASS_CONSISTENT)
    d.stream = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    return d, (atoms, Z)


def prolong(Xc, Nc: int):
    """Q1 prolongation of the device block Xc (Nc^3 x p, FP64 or FP32) to the
    grid with 2 Nc + 1 nodes per edge (ks_prolong), on the current stream."""
    import torch
    p = Xc.shape[1]
    Nf = 2 * Nc + 1
    out = torch.empty((Nf ** 3, p), dtype=Xc.dtype, device=Xc.device)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    lib = load_library()
    if Xc.dtype == torch.float64:
        _check(lib.ks_prolong(Nc, p, _ptr(Xc), _ptr(out), st))
    else:
        _check(lib.ks_prolong_f32(Nc, p, _ptr32(Xc), _ptr32(out), st))
    return out


def selftest_wait_timeout(stream=None) -> tuple[int, float]:
    """Run the bounded-wait probe (ks_selftest_wait_timeout): a grid-barrier
    wait that cannot complete.  Returns (recorded status, seconds)."""
    st = ctypes.c_int()
    sec = ctypes.c_double()
    s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    _check(load_library().ks_selftest_wait_timeout(s, ctypes.byref(st), ctypes.byref(sec)))
    return st.value, sec.value


def probe_fma(fp64: bool, blocks: int, iters: int, sink, stream=None) -> float:
    """Enqueue the FMA peak-rate probe (ks_probe_fma) on `stream` (a torch
    stream; default the current one); `sink` is a device float64 tensor of at
    least `blocks` entries.  Returns the launch's flop count; the caller
    times it."""
    import torch
    if sink.dtype != torch.float64 or not sink.is_cuda or sink.numel() < blocks:
        raise TypeError("sink must be a CUDA float64 tensor with at least `blocks` entries")
    st = (stream or torch.cuda.current_stream()).cuda_stream
    fl = ctypes.c_double()
    _check(load_library().ks_probe_fma(1 if fp64 else 0, blocks, iters, ctypes.c_void_p(st),
                                       _ptr(sink), ctypes.byref(fl)))
    return fl.value


def refine_grids(N: int, levels: int) -> list[int]:
    return [(N + 1) // (1 << (levels - 1 - l)) - 1 for l in range(levels)]


def minimize_refine(s, levels: int, x0: np.ndarray | None = None, coarse_gtol: float = 1e-3,
                    want_x: bool = True, **opts):
    """Alg. AdpConOptM with uniform refinement (ks_minimize_refine) for the
    ks_inputs.System `s`, ending on its own grid.  x0: the initial block on the
    coarsest grid (default: the seeded one drawn for that grid).  Returns
    (one result dict per level, the finest block or None)."""
    import torch
    grids = refine_grids(s.N, levels)
    if x0 is None:
        x0 = s.x0_for(grids[0])
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    d, keep = _system_desc(s, stream=torch.cuda.current_stream())
    o = default_opts(**opts)
    res = (Result * levels)()
    X = np.empty((s.N ** 3, s.p), dtype=np.float64) if want_x else None
    st = load_library().ks_minimize_refine(ctypes.byref(d), levels, x0.ctypes.data_as(_DP),
                                           ctypes.byref(o), coarse_gtol,
                                           X.ctypes.data_as(_DP) if want_x else None, res)
    if st not in (0, KS_ENOCONV):
        _check(st)
    return [result_dict(r) for r in res], X


class Problem:
    """One discretised KS system with its device workspace (ks_problem)."""

    def __init__(self, N: int, L: float, atoms, Z, p: int, rc: float = 0.5, occ: float = 2.0,
                 xc: int = KS_XC_SLATER_PZ81, cg_tol: float = 1e-10, cg_maxit: int = 20000,
                 stream=None, cg_precond: bool = True, kinetic: int = 0, mu: float = 1.0,
                 mass: int = 0):
        import torch
        lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        atoms = np.ascontiguousarray(np.asarray(atoms, dtype=np.float64).reshape(-1, 3))
        Z = np.ascontiguousarray(np.asarray(Z, dtype=np.float64).reshape(-1))
        self._atoms, self._Z = atoms, Z
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        d = ProblemDesc()
        d.N, d.L, d.natoms = N, L, len(Z)
        d.R = atoms.ctypes.data_as(_DP)
        d.Z = Z.ctypes.data_as(_DP)
        d.rc, d.p, d.occ, d.xc = rc, p, occ, xc
        d.cg_tol, d.cg_maxit, d.precision = cg_tol, cg_maxit, KS_FP64
        d.stream = ctypes.c_void_p(stream.cuda_stream)
        d.cg_precond = 1 if cg_precond else 0
        d.kinetic, d.mu, d.mass = kinetic, mu, mass
        self.desc = d
        h = ctypes.c_void_p()
        _check(lib.ks_problem_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.N, self.L, self.p, self.n = N, L, p, N ** 3
        self.h = L / (N + 1)

    @classmethod
    def from_system(cls, s, **kw) -> "Problem":
        kw.setdefault("kinetic", getattr(s, "kinetic", KS_KIN_ORBITALS))
        kw.setdefault("mu", getattr(s, "mu", 1.0))
        kw.setdefault("mass", getattr(s, "mass", KS_MASS_CONSISTENT))
        return cls(N=s.N, L=s.L, atoms=s.atoms, Z=s.Z, p=s.p, rc=s.rc, occ=s.occ, xc=s.xc, **kw)

    @staticmethod
    def bytes_for(N: int, p: int) -> int:
        d = ProblemDesc()
        d.N, d.L, d.natoms, d.rc, d.p, d.occ, d.xc = N, 1.0, 0, 0.5, p, 2.0, 0
        d.cg_tol, d.cg_maxit, d.precision = 1e-10, 100, KS_FP64
        return load_library().ks_problem_bytes(ctypes.byref(d))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load_library().ks_problem_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ helpers
    def empty_block(self):
        import torch
        return torch.empty((self.n, self.p), dtype=torch.float64, device="cuda")

    def empty_vec(self):
        import torch
        return torch.empty(self.n, dtype=torch.float64, device="cuda")

    # ------------------------------------------------------------ ks.h
    def energy_grad(self, X, want_ex: bool = True, want_d: bool = False):
        """(E, E_X or None, D or None, ||D||_M or None) at X."""
        E = ctypes.c_double()
        EX = self.empty_block() if want_ex else None
        D = self.empty_block() if want_d else None
        g = ctypes.c_double()
        _check(load_library().ks_energy_grad(self._h, _ptr(X), ctypes.byref(E), _ptr(EX), _ptr(D),
                                             ctypes.byref(g) if want_d else None))
        return E.value, EX, D, (g.value if want_d else None)

    def energy_parts(self) -> list[float]:
        a = (ctypes.c_double * 5)()
        _check(load_library().ks_energy_parts(self._h, a))
        return list(a)

    def retract(self, kind: int, X, EX, tau: float):
        out = self.empty_block()
        _check(load_library().ks_retract(self._h, kind, _ptr(X), _ptr(EX), tau, _ptr(out)))
        return out

    def orthonormalize(self, X):
        _check(load_library().ks_orthonormalize(self._h, _ptr(X)))
        return X

    def minimize(self, X, **opts) -> dict:
        """Alg. ConOptM in place on the device block X."""
        o = default_opts(**opts)
        r = Result()
        st = load_library().ks_minimize(self._h, _ptr(X), ctypes.byref(o), ctypes.byref(r))
        if st not in (KS_OK, KS_ENOCONV):
            _check(st)
        return result_dict(r)

    def minimize_host(self, X: np.ndarray, **opts) -> dict:
        """Alg. ConOptM on a host block (copied in and out inside the call)."""
        if not (X.dtype == np.float64 and X.flags["C_CONTIGUOUS"] and X.shape == (self.n, self.p)):
            raise TypeError("expected a C-contiguous float64 (n, p) array")
        o = default_opts(**opts)
        r = Result()
        st = load_library().ks_minimize_host(self._h, X.ctypes.data_as(_DP), ctypes.byref(o),
                                             ctypes.byref(r))
        if st not in (KS_OK, KS_ENOCONV):
            _check(st)
        return result_dict(r)

    def state_save(self) -> bytes:
        """Checkpoint of the last minimisation (host bytes)."""
        lib = load_library()
        nbytes = lib.ks_state_bytes(self._h)
        if nbytes == 0:
            raise KSError(KS_EINVAL, "no minimisation state to save")
        buf = ctypes.create_string_buffer(nbytes)
        _check(lib.ks_state_save(self._h, buf, nbytes))
        return buf.raw

    def state_load(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        _check(load_library().ks_state_load(self._h, buf, len(data)))

    # ------------------------------------------------------------ ks_steps.h
    def step_vext(self):
        out = self.empty_vec()
        _check(load_library().ks_step_vext(self._h, _ptr(out)))
        return out

    def step_eii(self) -> float:
        e = ctypes.c_double()
        _check(load_library().ks_step_eii(self._h, ctypes.byref(e)))
        return e.value

    def step_density(self, X):
        out = self.empty_vec()
        _check(load_library().ks_step_density(self._h, _ptr(X), _ptr(out)))
        return out

    def step_hartree(self, rho, vH=None, warm: bool = False):
        import torch
        v = torch.zeros_like(rho) if vH is None else vH
        r = torch.empty_like(rho)
        it = ctypes.c_int()
        _check(load_library().ks_step_hartree(self._h, _ptr(rho), _ptr(v), 1 if warm else 0,
                                              _ptr(r), ctypes.byref(it)))
        return v, r, it.value

    def step_potential(self, rho, vH, resid=None):
        veff = self.empty_vec()
        e = (ctypes.c_double * 4)()
        _check(load_library().ks_step_potential(self._h, _ptr(rho), _ptr(vH), _ptr(resid),
                                                _ptr(veff), e))
        return veff, list(e)

    def step_hamiltonian(self, X, veff, want_mx: bool = True):
        EX = self.empty_block()
        MX = self.empty_block() if want_mx else None
        k = ctypes.c_double()
        _check(load_library().ks_step_hamiltonian(self._h, _ptr(X), _ptr(veff), _ptr(EX), _ptr(MX),
                                                  ctypes.byref(k)))
        return EX, MX, k.value

    def step_hamiltonian_f32(self, X, veff, want_mx: bool = True):
        """FP32 stencil of the mixed phase: X float32 (n, p), veff float64 (n,)."""
        import torch
        EX = torch.empty((self.n, self.p), dtype=torch.float32, device="cuda")
        MX = torch.empty_like(EX) if want_mx else None
        k = ctypes.c_double()
        _check(load_library().ks_step_hamiltonian_f32(self._h, _ptr32(X), _ptr(veff), _ptr32(EX),
                                                      _ptr32(MX), ctypes.byref(k)))
        return EX, MX, k.value

    def step_mass(self, X):
        out = self.empty_block()
        _check(load_library().ks_step_mass(self._h, _ptr(X), _ptr(out)))
        return out

    def step_mass_inverse(self, E):
        out = self.empty_block()
        _check(load_library().ks_step_mass_inverse(self._h, _ptr(E), _ptr(out)))
        return out

    def step_gram(self, A, B):
        import torch
        pa, qb = A.shape[1], B.shape[1]
        out = torch.empty((pa, qb), dtype=torch.float64, device="cuda")
        _check(load_library().ks_step_gram(self._h, _ptr(A), pa, _ptr(B), qb, _ptr(out)))
        return out

    def set_tensor_cores(self, mode: int):
        """FP32-phase tensor cores: 0 never, 1 wide products (default), 2 always,
        3 wide products and the narrow updates (q <= 64, warp-specialised)."""
        _check(load_library().ks_set_tensor_cores(self._h, mode))

    def set_fp64_emulation(self, mode: int):
        """FP64 Grams on the tensor cores by digit splitting: 0 never, 1 wide, 2 always."""
        _check(load_library().ks_set_fp64_emulation(self._h, int(mode)))

    def set_tma(self, mode: int):
        """Stencil plane staging: 1 TMA ring (default, when aligned), 0 plain loads."""
        _check(load_library().ks_set_tma(self._h, mode))

    def step_gram_f32(self, A, B):
        """FP32 Gram of the mixed phase (A, B float32 CUDA tensors)."""
        import torch
        for t in (A, B):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise TypeError("expected contiguous torch.float32 CUDA tensors")
        pa, qb = A.shape[1], B.shape[1]
        out = torch.empty((pa, qb), dtype=torch.float64, device="cuda")
        _check(load_library().ks_step_gram_f32(self._h, A.data_ptr(), pa, B.data_ptr(), qb,
                                               _ptr(out)))
        return out

    def step_combine_f32(self, A1, C1, A2=None, C2=None, alpha: float = 1.0, beta: float = 0.0,
                         Bm=None):
        """FP32 update of the mixed phase (A1, A2, Bm float32; C1, C2 float64)."""
        import torch
        q = C1.shape[1]
        out = torch.empty((A1.shape[0], q), dtype=torch.float32, device="cuda")
        ptr = lambda t: None if t is None else t.data_ptr()
        _check(load_library().ks_step_combine_f32(
            self._h, ptr(A1), A1.shape[1], _ptr(C1), ptr(A2), A2.shape[1] if A2 is not None else 0,
            _ptr(C2), alpha, beta, ptr(Bm), ptr(out), q))
        return out

    def step_combine(self, A1, C1, A2=None, C2=None, alpha: float = 1.0, beta: float = 0.0, Bm=None):
        import torch
        q = C1.shape[1]
        out = torch.empty((A1.shape[0], q), dtype=torch.float64, device="cuda")
        _check(load_library().ks_step_combine(
            self._h, _ptr(A1), A1.shape[1], _ptr(C1), _ptr(A2), A2.shape[1] if A2 is not None else 0,
            _ptr(C2), alpha, beta, _ptr(Bm), _ptr(out), q))
        return out


class Server:
    """Continuous-batching job server (ks_server): submit systems as they
    arrive, collect results; admission is bounded by an HBM budget and a
    number of concurrent slots."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.ks_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(h)))
        self._h = h

    def submit(self, s, x0: np.ndarray | None = None, **opts) -> int:
        """Queue the ks_inputs.System `s` (initial block s.x0() unless given)."""
        x0 = np.ascontiguousarray(s.x0() if x0 is None else x0, dtype=np.float64)
        d, keep = _system_desc(s)
        o = default_opts(**opts)
        jid = ctypes.c_uint64()
        _check(load_library().ks_server_submit(self._h, ctypes.byref(d), ctypes.byref(o),
                                               x0.ctypes.data_as(_DP), ctypes.byref(jid)))
        return int(jid.value)

    def poll(self, job_id: int, wait: bool = True, want_x: bool = False, n: int = 0, p: int = 0):
        """None while running (wait=False); else (result dict, X or None, latency s)."""
        r = Result()
        lat = ctypes.c_double()
        X = np.empty((n, p), dtype=np.float64) if want_x else None
        st = load_library().ks_server_poll(self._h, job_id, 1 if wait else 0, ctypes.byref(r),
                                           X.ctypes.data_as(_DP) if want_x else None,
                                           ctypes.byref(lat))
        if st == KS_EAGAIN:
            return None
        _check(st)
        return result_dict(r), X, lat.value

    def stats(self) -> dict:
        st = ServerStats()
        _check(load_library().ks_server_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load_library().ks_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["Server", "Problem", "KSError", "load_library", "library_path", "default_opts",
           "KS_QR", "KS_CAYLEY", "KS_XC_SLATER", "KS_XC_SLATER_PZ81", "SIGNATURES"]


class Batch:
    """Job table of independent systems minimised together (ks_batch): every
    kernel launch of an iteration covers all jobs still iterating."""

    def __init__(self, systems, stream=None):
        lib = load_library()
        self.systems = list(systems)
        n = len(self.systems)
        descs = (ProblemDesc * n)()
        self._keep = []
        for j, s in enumerate(self.systems):
            descs[j], keep = _system_desc(s)
            self._keep.append(keep)
        h = ctypes.c_void_p()
        st = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        _check(lib.ks_batch_create(descs, n, st, ctypes.byref(h)))
        self._h = h

    @property
    def bytes(self) -> int:
        return load_library().ks_batch_bytes(self._h)

    def autotune(self) -> dict:
        """Time the candidate launch shapes on this job table and keep the fastest."""
        out = (_I * 4)()
        _check(load_library().ks_batch_autotune(self._h, out))
        return {"gram_rows": out[0], "comb_per_thread": out[1], "pot_per_thread": out[2],
                "stencil_planes": out[3]}

    def set_graphs(self, enable: bool):
        """Replay the step sequences as CUDA graphs (default) or launch them plainly."""
        _check(load_library().ks_batch_set_graphs(self._h, 1 if enable else 0))

    def minimize(self, X0=None, **opts):
        """Minimise every job from X0[j] (default s.x0()); returns (list of
        result dicts, list of final X arrays).  A job that did not converge
        has status KS_ENOCONV in its result; no exception is raised for it."""
        n = len(self.systems)
        X = [np.ascontiguousarray(s.x0() if X0 is None else X0[j], dtype=np.float64).copy()
             for j, s in enumerate(self.systems)]
        ptrs = (_DP * n)(*[x.ctypes.data_as(_DP) for x in X])
        res = (Result * n)()
        o = default_opts(**opts)
        st = load_library().ks_batch_minimize(self._h, ptrs, ctypes.byref(o), res)
        if st not in (KS_OK, KS_ENOCONV):
            _check(st)
        return [result_dict(r) for r in res], X

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load_library().ks_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
