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
