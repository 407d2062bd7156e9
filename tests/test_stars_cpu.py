"""Stars of the q-grid (fp_star_table, host code of the library; no GPU): the library's star map against an
orbit enumeration written here with numpy, and its rejection of operations that do not map the grid."""
import numpy as np
import pytest

from paper_2104_04895_gb300 import binding, synth


def orbits_numpy(grid, ops):
    """Representative (smallest index) of each grid point's orbit under ops and q -> -q, by breadth-first
    enumeration of each orbit."""
    grid = np.asarray(grid)
    mats = [np.asarray(R) for R in ops] + [np.eye(3, dtype=int)]
    mats = mats + [-R for R in mats]
    N = int(np.prod(grid))
    index = lambda g: int((g[0] * grid[1] + g[1]) * grid[2] + g[2])
    rep = -np.ones(N, dtype=int)
    for q in range(N):
        if rep[q] >= 0:
            continue
        g0 = np.array(np.unravel_index(q, tuple(grid)))
        orbit, todo = {q}, [g0]
        while todo:
            g = todo.pop()
            for R in mats:
                h = (R @ g) % grid
                k = index(h)
                if k not in orbit:
                    orbit.add(k)
                    todo.append(h)
        for k in orbit:
            rep[k] = min(orbit)
    return rep, len(np.unique(rep))


@pytest.mark.parametrize("maker,grid", [(lambda g: synth.simple_cubic(g, symmetric=True), (4, 4, 4)),
                                        (lambda g: synth.simple_cubic(g, symmetric=True), (6, 6, 6)),
                                        (lambda g: synth.diamond_si(g, symmetric=True), (4, 4, 4)),
                                        (lambda g: synth.diamond_si(g, symmetric=True), (5, 5, 5))])
def test_star_table_matches_orbit_enumeration(maker, grid):
    cr = maker(grid)
    ops = synth.point_group_ops(cr)
    rep, n = binding.star_table(cr.grid, ops)
    ref, nref = orbits_numpy(cr.grid, ops)
    assert n == nref
    assert np.array_equal(rep, ref)
    # every representative is its own representative and the smallest index of its star
    assert np.all(rep[rep] == rep) and np.all(rep <= np.arange(len(rep)))


def test_star_counts_of_the_cubic_group():
    """Counts by hand: under O_h a point of the Gamma-centred n x n x n simple-cubic grid is fixed by its
    coordinates' absolute values (g and n - g are equivalent) up to order, i.e. a multiset of three values in
    0 .. n/2: C(n/2 + 3, 3) stars, 10 for n = 4 and 20 for n = 6."""
    ops = synth.point_group_ops(synth.simple_cubic((4, 4, 4), symmetric=True))
    assert binding.star_table((4, 4, 4), ops)[1] == 10
    assert binding.star_table((6, 6, 6), ops)[1] == 20
    # time reversal alone pairs q with -q: (N^3 + number of self-conjugate points) / 2
    assert binding.star_table((4, 4, 4), np.zeros((0, 3, 3), np.int32))[1] == (64 + 8) // 2


def test_star_table_rejects_bad_operations():
    with pytest.raises(binding.FourPhononError):
        binding.star_table((4, 4, 4), np.array([[[2, 0, 0], [0, 1, 0], [0, 0, 1]]]))  # not unimodular
    with pytest.raises(binding.FourPhononError):
        binding.star_table((4, 4, 2), np.array([[[0, 0, 1], [0, 1, 0], [1, 0, 0]]]))  # mixes axes of 4 and 2
