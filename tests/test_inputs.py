"""Pins of the seeded input recipes against what the paper prints, and of
host-side helpers that need no GPU."""
import os

import ks_inputs as ki
from oracle import stiefel as ost

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_fcc_clusters_have_the_papers_atom_counts():
    # Table compare-OF: 365, 1688, 4631 and 7813 aluminium atoms for blocks of
    # 4, 7, 10 and 12 fcc cells per edge
    rows = []
    with open(os.path.join(GOLDEN, "of_cluster_atoms.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                cells, atoms = line.split()
                rows.append((int(cells), int(atoms)))
    assert len(rows) == 4
    for cells, atoms in rows:
        s = ki.config_of_al(cells=cells)
        assert len(s.atoms) == atoms
        assert s.occ == 3.0 * atoms and s.p == 1 and s.kinetic == 1 and s.mass == 1
        # every atom inside the box with 6 bohr of vacuum on each side, to within
        # the half grid spacing by which the box is rounded to the grid
        tol = 0.5 * s.h + 1e-9
        assert s.atoms.min() >= 6.0 - tol and s.atoms.max() <= s.L - 6.0 + tol


def test_refinement_grids_match_the_oracle():
    # the binding's helper is pure Python: importing the package loads no
    # device code
    import paper_1308_2864_gb300 as ks
    for N, levels in [(15, 3), (159, 2), (255, 4), (11, 1)]:
        assert ks.refine_grids(N, levels) == ost.refine_levels(N, levels)


def test_splitmix64_known_outputs():
    # splitmix64 (Steele, Lea and Flood, OOPSLA 2014): the first outputs of
    # the generator from state 1234567, and from state 0, as the public-domain
    # reference implementation prints them
    g = ki.SplitMix64(1234567)
    assert [g.next_u64() for _ in range(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]
    assert ki.SplitMix64(0).next_u64() == 0xE220A8397B1DCDAF


def test_vectorised_stream_equals_the_scalar_one():
    # uniform_block (numpy, wrapping uint64) and SplitMix64.uniform (Python
    # integers, masked) give the same doubles, from any offset
    key = ki.stream_key(1001, 7, ki.STREAM_X0)
    g = ki.SplitMix64(key)
    scalar = [g.uniform() for _ in range(300)]
    assert list(ki.uniform_block(key, 300)) == scalar
    assert list(ki.uniform_block(key, 100, start=200)) == scalar[200:]
    assert all(0.0 <= u < 1.0 for u in scalar)


def _min_separation(atoms):
    import numpy as np
    d = np.linalg.norm(atoms[:, None, :] - atoms[None, :, :], axis=-1)
    d[np.diag_indices(len(atoms))] = np.inf
    return d.min()


def test_single_system_recipes():
    # the configurations the bench and the parity tests use: grids, atom
    # placement, charges (2 p electrons = sum Z) and functionals
    import numpy as np
    c1 = ki.config_c1()
    assert (c1.N, c1.L, c1.p, c1.xc, c1.retraction) == (24, 10.0, 4, 0, "cayley")
    assert c1.h == 0.4 and len(c1.atoms) == 2
    assert c1.atoms.min() >= 2.5 and c1.atoms.max() <= 7.5
    assert _min_separation(c1.atoms) >= 1.5
    for c, (N, L, grid, p) in ((ki.config_c2(), (64, 20.0, (4, 4, 2), 64)),
                               (ki.config_c3(), (128, 40.0, (8, 8, 4), 512))):
        assert (c.N, c.L, c.p, c.xc, c.retraction) == (N, L, p, 1, "qr")
        assert len(c.atoms) == np.prod(grid) and 2 * c.p == c.Z.sum()
        # every atom within 0.3 bohr (per axis) of its own simple-cubic site
        sites = np.array([((i + 0.5) * L / grid[0], (j + 0.5) * L / grid[1],
                           (l + 0.5) * L / grid[2])
                          for i in range(grid[0]) for j in range(grid[1]) for l in range(grid[2])])
        assert np.abs(c.atoms - sites).max() <= 0.3
    for c in (c1, ki.config_c2(), ki.config_c3()):
        assert c.rc == 0.5 and c.occ == 2.0 and np.all(c.Z == 4.0)


def test_job_stream_recipes():
    import numpy as np
    jobs = ki.config_c4_jobs()
    assert len(jobs) == 256
    Ns = np.array([s.N for s in jobs])
    assert Ns.min() >= 20 and Ns.max() <= 48 and len(set(Ns)) > 15
    for s in jobs:
        natoms = len(s.atoms)
        assert 2 <= natoms <= 16 and s.p == 2 * natoms and s.L == 0.4 * (s.N + 1)
        assert s.atoms.min() >= 1.5 and s.atoms.max() <= s.L - 1.5
        assert _min_separation(s.atoms) >= 0.8
    stream = ki.config_c5_jobs()
    for s in stream:
        assert 24 <= s.N <= 96 and 8 <= s.p <= 128 and s.p % 2 == 0
        assert len(s.atoms) == s.p // 2
    # the same seed gives the same jobs
    again = ki.config_c4_jobs(njobs=3)
    assert all(np.array_equal(a.atoms, b.atoms) for a, b in zip(again, jobs[:3]))
    t = ki.poisson_arrivals(1004, 2000, rate=4.0)
    assert np.all(np.diff(t) > 0)
    assert abs(len(t) / t[-1] - 4.0) < 0.4                   # mean rate
