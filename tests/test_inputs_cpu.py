"""The seeded synthetic inputs obey the symmetries their recipe states (Sec. 2.3).

* Phi4 quartet lists are invariant under permutations of their four (atom, cell, Cartesian) legs (Eq. TS), in both
  the bond-energy form and the general form used by the index-order parity tests.
* The bond-energy Phi4 obeys the acoustic sum rule in every leg (Eq. ASR); the general form does not, as stated.
* Phi2 obeys the acoustic sum rule and the pair symmetry Phi2(0i; Rj)_ab = Phi2(0j; -R i)_ba.
* Phi3 is invariant under permutations of its three legs and obeys the acoustic sum rule.
"""
import itertools

import numpy as np
import pytest

from paper_2104_04895_gb300 import synth

MAKERS = [
    ("simple-cubic", lambda **k: synth.simple_cubic((2, 2, 2), **k)),
    ("diamond", lambda **k: synth.diamond_si((2, 2, 2), **k)),
    ("zincblende", lambda **k: synth.zincblende_bas((2, 2, 2), **k)),
    ("licoo2", lambda **k: synth.licoo2((2, 2, 2), **k)),
]


def quartet_table(idx, val, order):
    """{(atoms, cells of legs 2..order): tensor} with the first leg in cell 0."""
    table = {}
    for row, v in zip(idx, val):
        atoms = tuple(int(a) for a in row[:order])
        cells = tuple(tuple(int(c) for c in row[order + 3 * m: order + 3 * m + 3]) for m in range(order - 1))
        key = (atoms, cells)
        assert key not in table
        table[key] = v.reshape((3,) * order)
    return table


def legs(key):
    atoms, cells = key
    return [(atoms[0], (0, 0, 0))] + [(a, c) for a, c in zip(atoms[1:], cells)]


def rebased(sites):
    c0 = np.array(sites[0][1])
    return (tuple(s[0] for s in sites), tuple(tuple(int(x) for x in np.array(s[1]) - c0) for s in sites[1:]))


def check_permutation_symmetry(table, order):
    scale = max(np.abs(t).max() for t in table.values())
    for key, T in table.items():
        sites = legs(key)
        for p in itertools.permutations(range(order)):
            other = rebased([sites[i] for i in p])
            assert other in table, (key, p)
            assert np.abs(table[other] - np.transpose(T, p)).max() <= 1e-12 * scale, (key, p)


def check_sum_rule(table, order):
    """Summing over the atom and cell of the last leg gives zero for every other leg and Cartesian index."""
    scale = max(np.abs(t).max() for t in table.values())
    acc = {}
    for key, T in table.items():
        atoms, cells = key
        rest = (atoms[:-1], cells[:-1])
        acc[rest] = acc.get(rest, 0.0) + T
    worst = max(np.abs(s).max() for s in acc.values())
    return worst / scale


@pytest.mark.parametrize("name,maker", MAKERS, ids=[m[0] for m in MAKERS])
def test_phi4_transposition_symmetry_and_sum_rule(name, maker):
    cr = maker()
    table = quartet_table(cr.fc4_idx, cr.fc4_val, 4)
    check_permutation_symmetry(table, 4)
    assert check_sum_rule(table, 4) <= 1e-12
    gen = maker(general=True)
    gtable = quartet_table(gen.fc4_idx, gen.fc4_val, 4)
    assert set(gtable) == set(table)          # the same quartets, other values
    check_permutation_symmetry(gtable, 4)
    assert check_sum_rule(gtable, 4) > 1e-3  # the general form does not obey the sum rule
    # and its Cartesian indices are not symmetric within one quartet, which the bond-energy form's are
    asym = max(np.abs(T - T.transpose(1, 0, 2, 3)).max() for T in gtable.values())
    sym = max(np.abs(T - T.transpose(1, 0, 2, 3)).max() for T in table.values())
    assert asym > 1.0 and sym <= 1e-12 * max(np.abs(T).max() for T in table.values())


@pytest.mark.parametrize("name,maker", MAKERS, ids=[m[0] for m in MAKERS])
def test_phi3_transposition_symmetry_and_sum_rule(name, maker):
    cr = maker()
    table = quartet_table(cr.fc3_idx, cr.fc3_val, 3)
    check_permutation_symmetry(table, 3)
    assert check_sum_rule(table, 3) <= 1e-12


@pytest.mark.parametrize("name,maker", MAKERS, ids=[m[0] for m in MAKERS])
def test_phi2_sum_rule_and_pair_symmetry(name, maker):
    cr = maker()
    blocks = {}
    for row, v in zip(cr.fc2_idx, cr.fc2_val):
        key = (int(row[0]), int(row[1]), tuple(int(c) for c in row[2:5]))
        blocks[key] = blocks.get(key, 0.0) + v.reshape(3, 3)
    scale = max(np.abs(b).max() for b in blocks.values())
    for i in range(cr.natoms):
        s = sum(b for (a, _, _), b in blocks.items() if a == i)
        assert np.abs(s).max() <= 1e-12 * scale
    for (i, j, R), b in blocks.items():
        back = blocks.get((j, i, tuple(-c for c in R)))
        assert back is not None and np.abs(back - b.T).max() <= 1e-12 * scale
