"""Pins of the oracle's stencils against the paper (Sec. 2, big stencil S
and sub-stencils S_m) and against the symmetry of the cube."""
import itertools
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _printed_substencils():
    rows = {}
    with open(os.path.join(GOLDEN, "substencils_printed.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            rows[int(parts[0])] = [tuple(int(x) for x in p.split(",")) for p in parts[1:]]
    return rows


def test_big_stencil_is_block_minus_corners():
    big, _ = oracle.stencils()
    cells = {tuple(int(x) for x in r) for r in big}
    assert len(cells) == 18
    expect = {o for o in itertools.product((-1, 0, 1), repeat=3)
              if o != (0, 0, 0) and abs(o[0] * o[1] * o[2]) != 1}
    assert cells == expect


def test_substencils_match_printed_ones():
    _, sub = oracle.stencils()
    printed = _printed_substencils()
    for m in (1, 2, 3, 5, 6, 7):
        assert [tuple(int(x) for x in r) for r in sub[m - 1]] == printed[m]
    # Reading of the printed S4, S8: the diagonal (-1,-1,0) is kept and the
    # two in-plane axis cells are those adjacent to it.
    for m in (4, 8):
        got = [tuple(int(x) for x in r) for r in sub[m - 1]]
        assert got[2] == printed[m][2] == (-1, -1, 0)
        assert got[0] == (-1, 0, 0) and got[1] == (0, -1, 0)
        assert got[3] == printed[m][3]


def test_substencils_inside_big_stencil_and_distinct():
    big, sub = oracle.stencils()
    bigset = {tuple(int(x) for x in r) for r in big}
    sets = set()
    for m in range(24):
        cells = [tuple(int(x) for x in r) for r in sub[m]]
        assert len(set(cells)) == 4
        assert set(cells) <= bigset
        # three independent directions: the 4x3 system has rank 3
        assert np.linalg.matrix_rank(np.array(cells, dtype=float)) == 3
        sets.add(frozenset(cells))
    assert len(sets) == 24


def test_substencil_family_invariant_under_cube_symmetries():
    """'Symmetrically, another two thirds...': the 24 sub-stencils form one
    orbit family closed under the 48 rotations/reflections of the cube."""
    _, sub = oracle.stencils()
    fam = {frozenset(tuple(int(x) for x in r) for r in sub[m]) for m in range(24)}
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((-1, 1), repeat=3):
            img = set()
            for s in fam:
                img.add(frozenset(tuple(signs[d] * c[perm[d]] for d in range(3)) for c in s))
            assert img == fam
