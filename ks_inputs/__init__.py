"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle and the bench.

This module holds no arithmetic of the method: it only draws random numbers
(a counter-based splitmix64 stream), places pseudo-atoms and fills the initial
orbital block X0.  Everything that depends on the discretisation (the mass
matrix, M-orthonormalisation, potentials) lives on each side separately.

Workload recipes (the synthetic stand-ins for the paper's molecules, which
need geometries and pseudopotentials that are not available):

  * ``c1``  cube side 10 bohr, 24^3 interior Q1 nodes, 2 atoms (Z=4) drawn
            uniformly in [L/4, 3L/4]^3 with a 1.5 bohr minimum separation,
            p=4 doubly occupied orbitals, Slater exchange only, Cayley step.
  * ``c2``  cube side 20 bohr, 64^3 nodes, 32 atoms on a 4x4x2 simple lattice
            jittered by U(-0.3, 0.3) bohr, p=64, Slater + PZ81, QR step.
  * ``c3``  cube side 40 bohr, 128^3 nodes, 256 atoms on 8x8x4, p=512.
  * ``c4``  256 jobs, N = round(exp(U(ln 20, ln 48))), spacing 0.4 bohr,
            2..16 atoms placed uniformly in [1.5, L-1.5]^3, p = 2 * atoms.
  * ``of``  orbital-free (Thomas-Fermi-von Weizsaecker) aluminium-like
            clusters: the sites of an s x s x s block of face-centred cubic
            cells (cube edge 7.559 bohr, every corner and face centre of the
            block), Z = 3 pseudo-atoms, 6 bohr of vacuum on each side, grid
            spacing about 0.4 bohr, one "orbital" (p = 1) occupied by all
            3 * atoms electrons, lumped mass (h^3 I), initial guess
            1 + 0.1 U(-1, 1) per node.

The grid has N interior nodes per edge and spacing h = L/(N+1); interior
node (ix, iy, iz) sits at ((ix+1)h, (iy+1)h, (iz+1)h) and has flat index
k = (iz*N + iy)*N + ix.  X is stored row-major n x p (orbital index fastest).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN_GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1

# Stream ids inside one (seed, job) key.
STREAM_ATOMS = 0
STREAM_X0 = 1
STREAM_JOBSIZE = 2
STREAM_ARRIVALS = 3
STREAM_SUBSAMPLE = 4


def _mix64(z: int) -> int:
    """splitmix64 output function (Steele, Lea, Flood 2014)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, job: int, stream: int) -> int:
    """Initial splitmix64 state for one named stream of one job."""
    return _mix64((seed * 0x100000001B3) ^ (job * 0x10001) ^ (stream << 56))


class SplitMix64:
    """Counter-based splitmix64: the i-th output (i = 0, 1, ...) is
    mix64(key + (i+1)*GOLDEN_GAMMA)."""

    def __init__(self, key: int):
        self.key = key & MASK64
        self.count = 0

    def next_u64(self) -> int:
        self.count += 1
        return _mix64(self.key + self.count * GOLDEN_GAMMA)

    def uniform(self) -> float:
        """Double in [0, 1): top 53 bits times 2^-53."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)


def uniform_block(key: int, count: int, start: int = 0) -> np.ndarray:
    """Vectorised outputs start..start+count-1 of the stream `key` as doubles
    in [0, 1)."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + idx * np.uint64(GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def initial_orbitals(seed: int, job: int, n: int, p: int) -> np.ndarray:
    """X0 with entries U(-1, 1), filled in row-major order (node-major,
    orbital fastest).  Not yet M-orthonormal."""
    u = uniform_block(stream_key(seed, job, STREAM_X0), n * p)
    return (2.0 * u - 1.0).reshape(n, p)


def initial_density_amplitude(seed: int, job: int, n: int) -> np.ndarray:
    """Orbital-free start: a nearly uniform amplitude 1 + 0.1 U(-1, 1) per
    node (n x 1).  Not yet M-normalised."""
    u = uniform_block(stream_key(seed, job, STREAM_X0), n)
    return (1.0 + 0.1 * (2.0 * u - 1.0)).reshape(n, 1)


@dataclass
class System:
    """One synthetic Kohn-Sham system (geometry and sizes only)."""
    N: int                      # interior nodes per edge
    L: float                    # cube side (bohr)
    atoms: np.ndarray           # (natoms, 3) positions in bohr
    Z: np.ndarray               # (natoms,) valence charges
    p: int                      # number of orbitals
    xc: int = 0                 # 0 = Slater exchange, 1 = Slater + PZ81
    rc: float = 0.5             # erf smearing radius of the pseudo-atom
    occ: float = 2.0            # occupation per orbital
    retraction: str = "qr"      # "qr" or "cayley"
    kinetic: int = 0            # 0 = orbitals, (f/2) tr(X^T K X); 1 = TFW density functional (p = 1)
    mass: int = 0               # 0 = consistent Q1 mass matrix; 1 = lumped (h^3 I)
    mu: float = 1.0             # weight of the von Weizsaecker term (kinetic = 1)
    seed: int = 0
    job: int = 0
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def h(self) -> float:
        return self.L / (self.N + 1)

    @property
    def n(self) -> int:
        return self.N ** 3

    def x0(self) -> np.ndarray:
        return self.x0_for(self.N)

    def x0_for(self, N: int) -> np.ndarray:
        """The seeded initial block drawn for an N^3 grid (the coarsest grid of
        a refinement run)."""
        if self.kinetic == 1:
            return initial_density_amplitude(self.seed, self.job, N ** 3)
        return initial_orbitals(self.seed, self.job, N ** 3, self.p)


def _random_atoms(rng: SplitMix64, natoms: int, lo: float, hi: float,
                  dmin: float, relaxed: float, tries: int = 10_000) -> np.ndarray:
    pos: list[tuple[float, float, float]] = []
    for _ in range(natoms):
        limit = dmin
        t = 0
        while True:
            cand = tuple(lo + (hi - lo) * rng.uniform() for _ in range(3))
            if all(math.dist(cand, q) >= limit for q in pos):
                pos.append(cand)
                break
            t += 1
            if t == tries:
                limit = relaxed
    return np.array(pos, dtype=np.float64).reshape(natoms, 3)


def _lattice_atoms(rng: SplitMix64, L: float, nx: int, ny: int, nz: int,
                   jitter: float) -> np.ndarray:
    pos = []
    for i in range(nx):
        for j in range(ny):
            for l in range(nz):
                site = ((i + 0.5) * L / nx, (j + 0.5) * L / ny, (l + 0.5) * L / nz)
                pos.append(tuple(s + jitter * (2.0 * rng.uniform() - 1.0) for s in site))
    return np.array(pos, dtype=np.float64)


def config_c1(seed: int = 1000) -> System:
    L, N = 10.0, 24
    rng = SplitMix64(stream_key(seed, 0, STREAM_ATOMS))
    atoms = _random_atoms(rng, 2, L / 4, 3 * L / 4, 1.5, 1.5)
    return System(N=N, L=L, atoms=atoms, Z=np.full(2, 4.0), p=4, xc=0,
                  retraction="cayley", seed=seed, name="c1: 24^3 grid, 2 atoms, p=4, FP64 Cayley")


def config_c2(seed: int = 1001) -> System:
    L, N = 20.0, 64
    rng = SplitMix64(stream_key(seed, 0, STREAM_ATOMS))
    atoms = _lattice_atoms(rng, L, 4, 4, 2, 0.3)
    return System(N=N, L=L, atoms=atoms, Z=np.full(32, 4.0), p=64, xc=1,
                  retraction="qr", seed=seed, name="c2: 64^3 grid, 32 atoms, p=64, QR")


def config_c3(seed: int = 1002) -> System:
    L, N = 40.0, 128
    rng = SplitMix64(stream_key(seed, 0, STREAM_ATOMS))
    atoms = _lattice_atoms(rng, L, 8, 8, 4, 0.3)
    return System(N=N, L=L, atoms=atoms, Z=np.full(256, 4.0), p=512, xc=1,
                  retraction="qr", seed=seed, name="c3: 128^3 grid, 256 atoms, p=512, QR")


def config_c4_jobs(seed: int = 1003, njobs: int = 256) -> list[System]:
    jobs = []
    for j in range(njobs):
        rng = SplitMix64(stream_key(seed, j, STREAM_JOBSIZE))
        N = int(round(math.exp(math.log(20) + (math.log(48) - math.log(20)) * rng.uniform())))
        natoms = 2 + int(15 * rng.uniform())          # U{2..16}
        L = 0.4 * (N + 1)
        arng = SplitMix64(stream_key(seed, j, STREAM_ATOMS))
        atoms = _random_atoms(arng, natoms, 1.5, L - 1.5, 1.2, 0.8)
        jobs.append(System(N=N, L=L, atoms=atoms, Z=np.full(natoms, 4.0), p=2 * natoms,
                           xc=1, retraction="qr", seed=seed, job=j,
                           name=f"c4 job {j}: {N}^3, {natoms} atoms"))
    return jobs


def config_c5_jobs(seed: int = 1004, njobs: int = 512) -> list[System]:
    """Serving stream: N log-uniform in [24, 96] (spacing 0.4 bohr), p
    log-uniform in [8, 128] rounded to an even number, p/2 atoms (Z = 4)
    placed like c4."""
    jobs = []
    for j in range(njobs):
        rng = SplitMix64(stream_key(seed, j, STREAM_JOBSIZE))
        N = int(round(math.exp(math.log(24) + (math.log(96) - math.log(24)) * rng.uniform())))
        p = int(round(math.exp(math.log(8) + (math.log(128) - math.log(8)) * rng.uniform()) / 2)) * 2
        p = min(max(p, 8), 128)
        natoms = p // 2
        L = 0.4 * (N + 1)
        arng = SplitMix64(stream_key(seed, j, STREAM_ATOMS))
        atoms = _random_atoms(arng, natoms, 1.5, L - 1.5, 1.2, 0.8)
        jobs.append(System(N=N, L=L, atoms=atoms, Z=np.full(natoms, 4.0), p=p, xc=1,
                           retraction="qr", seed=seed, job=j,
                           name=f"c5 job {j}: {N}^3, p={p}"))
    return jobs


def poisson_arrivals(seed: int, njobs: int, rate: float) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with the given rate (jobs/s):
    cumulative exponential gaps -ln(1-u)/rate from the arrivals stream."""
    u = uniform_block(stream_key(seed, 0, STREAM_ARRIVALS), njobs)
    return np.cumsum(-np.log1p(-u) / rate)


def stream_subsample(k: int, njobs: int = 512, seed: int = 1004) -> list[int]:
    """k distinct indices of a stream of njobs jobs, in increasing order: a
    seeded partial Fisher-Yates shuffle (swap position i with a uniform pick
    among i .. njobs - 1, for i < k).  The jobs a slower form runs in place
    of the whole stream; k >= njobs gives every index."""
    if k >= njobs:
        return list(range(njobs))
    idx = list(range(njobs))
    rng = SplitMix64(stream_key(seed, 0, STREAM_SUBSAMPLE))
    for i in range(max(k, 0)):
        j = i + int(rng.uniform() * (njobs - i))
        idx[i], idx[j] = idx[j], idx[i]
    return sorted(idx[:max(k, 0)])


def small_system(N: int = 6, L: float = 6.0, natoms: int = 1, p: int = 2,
                 xc: int = 1, seed: int = 7, retraction: str = "qr",
                 Z: float | None = None) -> System:
    """A tiny system for brute-force checks (atoms placed like c4)."""
    rng = SplitMix64(stream_key(seed, 0, STREAM_ATOMS))
    lo, hi = 0.3 * L, 0.7 * L
    atoms = _random_atoms(rng, natoms, lo, hi, 1.2, 0.8)
    zval = float(2 * p) / natoms if Z is None else Z
    return System(N=N, L=L, atoms=atoms, Z=np.full(natoms, zval), p=p, xc=xc,
                  retraction=retraction, seed=seed, name=f"small {N}^3 p={p}")


def fcc_cluster_sites(cells: int, a: float) -> np.ndarray:
    """Sites of an s x s x s block of face-centred cubic cells with cube
    edge a: every lattice point (corners and face centres) inside the block,
    boundary included, with the block's corner at the origin."""
    pts = set()
    m = 2 * cells
    for i in range(m + 1):
        for j in range(m + 1):
            for l in range(m + 1):
                if (i + j + l) % 2 == 0:
                    pts.add((i, j, l))
    return np.array(sorted(pts), dtype=np.float64) * (0.5 * a)


def config_of_al(cells: int = 4, seed: int = 1010, spacing: float = 0.4,
                 margin: float = 6.0, mu: float = 1.0, N: int | None = None) -> System:
    """Orbital-free aluminium-like cluster (see the module docstring).  With N
    given, the grid has N interior nodes per edge and the spacing follows."""
    a = 7.559
    sites = fcc_cluster_sites(cells, a)
    L0 = cells * a + 2.0 * margin
    if N is None:
        N = int(round(L0 / spacing)) - 1
        L = spacing * (N + 1)
    else:
        L = L0
    atoms = sites + 0.5 * (L - cells * a)
    natoms = len(atoms)
    return System(N=N, L=L, atoms=atoms, Z=np.full(natoms, 3.0), p=1, xc=1, rc=1.15,
                  occ=3.0 * natoms, retraction="qr", kinetic=1, mu=mu, mass=1, seed=seed,
                  name=f"of: {cells}^3 fcc cells, {natoms} Al-like atoms, {N}^3 grid")


def small_of_system(N: int = 6, L: float = 6.0, natoms: int = 2, Z: float = 1.0,
                    seed: int = 11, mu: float = 1.0, xc: int = 1, mass: int = 1) -> System:
    """A tiny orbital-free system (p = 1, every electron in the one amplitude;
    lumped mass unless told otherwise)."""
    rng = SplitMix64(stream_key(seed, 0, STREAM_ATOMS))
    atoms = _random_atoms(rng, natoms, 0.3 * L, 0.7 * L, 1.2, 0.8)
    return System(N=N, L=L, atoms=atoms, Z=np.full(natoms, Z), p=1, xc=xc, rc=1.0,
                  occ=Z * natoms, retraction="cayley", kinetic=1, mu=mu, mass=mass, seed=seed,
                  name=f"small OF {N}^3")


CONFIGS = {"c1": config_c1, "c2": config_c2, "c3": config_c3}
