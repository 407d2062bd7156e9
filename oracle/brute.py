"""Brute-force supercell vertex on tiny grids (test infrastructure only; parity pin for Eq. V4).

The N1 x N2 x N3 grid is the Born-von Karman supercell of N cells.  Phi4 is folded
onto it (cell c of atom i, cells c+R_j, c+R_k, c+R_l wrapped), and each mode becomes
a supercell displacement pattern u(c, i) = e(i) exp(i q.R_c) / sqrt(M_i).  Then

  V = (1/N) sum_{I J K L} Phi_sc[I J K L] u_q(I) u_q'(J) u_q''(K) conj(u_q'''(L))

equals Eq. V4 of the paper when q''' = q + q' + q'' (mod G) and vanishes otherwise,
with no cell-phase convention, no quartet list and no reciprocal-space assembly.
"""
from __future__ import annotations

import itertools

import numpy as np


def supercell_phi4(cryst):
    grid = cryst.grid
    N = int(np.prod(grid))
    nat = cryst.natoms
    n = 3 * nat * N
    P = np.zeros((n, n, n, n))
    cells = list(itertools.product(range(grid[0]), range(grid[1]), range(grid[2])))

    def site(c, R, atom):
        cc = [(c[a] + int(R[a])) % grid[a] for a in range(3)]
        ci = (cc[0] * grid[1] + cc[1]) * grid[2] + cc[2]
        return 3 * (ci * nat + atom)

    for idx, val in zip(cryst.fc4_idx, cryst.fc4_val):
        i, j, k, l = (int(x) for x in idx[:4])
        Rj, Rk, Rl = idx[4:7], idx[7:10], idx[10:13]
        blk = val.reshape(3, 3, 3, 3)
        for c in cells:
            I = site(c, (0, 0, 0), i)
            J = site(c, Rj, j)
            K = site(c, Rk, k)
            L = site(c, Rl, l)
            P[I:I + 3, J:J + 3, K:K + 3, L:L + 3] += blk
    return P


def displacement(cryst, q, evec_q):
    """u[(cell, atom, alpha), branch] for grid point q (row-major index) and its eigenvectors (nb, nb)."""
    grid = cryst.grid
    N = int(np.prod(grid))
    nat = cryst.natoms
    gq = np.array([q // (grid[1] * grid[2]), (q // grid[2]) % grid[1], q % grid[2]], float)
    out = np.zeros((3 * nat * N, cryst.nb), complex)
    ci = 0
    for c in itertools.product(range(grid[0]), range(grid[1]), range(grid[2])):
        ph = np.exp(2j * np.pi * float(np.dot(gq / np.array(grid, float), np.array(c, float))))
        for a in range(nat):
            sl = slice(3 * (ci * nat + a), 3 * (ci * nat + a) + 3)
            out[sl, :] = (evec_q[:, 3 * a:3 * a + 3].T * ph) / np.sqrt(cryst.mass[a])
        ci += 1
    return out


def vertex(cryst, P, evec, q, q1, q2, q3, conj1=False, conj2=False):
    """V[j, j1, j2, j3] = (1/N) sum Phi_sc u_q u_q1 u_q2 conj(u_q3); conj flags give e^{-lambda} legs."""
    N = int(np.prod(cryst.grid))
    u0 = displacement(cryst, q, evec[q])
    u1 = displacement(cryst, q1, evec[q1])
    u2 = displacement(cryst, q2, evec[q2])
    u3 = displacement(cryst, q3, evec[q3])
    if conj1:
        u1 = u1.conj()
    if conj2:
        u2 = u2.conj()
    return np.einsum("IJKL,Ia,Jb,Kc,Ld->abcd", P, u0, u1, u2, u3.conj(), optimize=True) / N


def supercell_phi3(cryst):
    """Third-order force constants folded onto the Born-von Karman supercell (for Eq. V3)."""
    grid = cryst.grid
    N = int(np.prod(grid))
    nat = cryst.natoms
    n = 3 * nat * N
    P = np.zeros((n, n, n))
    cells = list(itertools.product(range(grid[0]), range(grid[1]), range(grid[2])))

    def site(c, R, atom):
        cc = [(c[a] + int(R[a])) % grid[a] for a in range(3)]
        ci = (cc[0] * grid[1] + cc[1]) * grid[2] + cc[2]
        return 3 * (ci * nat + atom)

    for idx, val in zip(cryst.fc3_idx, cryst.fc3_val):
        i, j, k = (int(x) for x in idx[:3])
        Rj, Rk = idx[3:6], idx[6:9]
        blk = val.reshape(3, 3, 3)
        for c in cells:
            P[site(c, (0, 0, 0), i):site(c, (0, 0, 0), i) + 3, site(c, Rj, j):site(c, Rj, j) + 3,
              site(c, Rk, k):site(c, Rk, k) + 3] += blk
    return P


def vertex3(cryst, P3, evec, q, q1, q2, conj1=False):
    """V[j, j1, j2] = (1/N) sum Phi3_sc u_q u_q1 conj(u_q2); conj1 gives the e^{-lambda'} leg."""
    N = int(np.prod(cryst.grid))
    u0 = displacement(cryst, q, evec[q])
    u1 = displacement(cryst, q1, evec[q1])
    u2 = displacement(cryst, q2, evec[q2])
    if conj1:
        u1 = u1.conj()
    return np.einsum("IJK,Ia,Jb,Kc->abc", P3, u0, u1, u2.conj(), optimize=True) / N
