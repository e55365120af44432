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
    import importlib.util
    spec = importlib.util.find_spec("paper_1308_2864_gb300")
    assert spec is not None
    # the binding's helper is pure Python (no library load)
    src = open(spec.origin).read()
    assert "def refine_grids" in src
    ns = {}
    exec(src[src.index("def refine_grids"):src.index("def minimize_refine")], ns)
    for N, levels in [(15, 3), (159, 2), (255, 4), (11, 1)]:
        assert ns["refine_grids"](N, levels) == ost.refine_levels(N, levels)
