"""A CPU model of the fluid-cell list layout, with the numbering and
neighbour-table rules of the library's context builder: fluid cells numbered
Block by Block in (z, y, x) order; for each cell and direction q = 1..18 the
list index of the pull source x - e_q (periodic images and Block faces
resolved), or -1 / -2 / -3 for a resting wall, moving wall or pressure node;
row 0 marking cells with a pressure link.  One list step (pull through the
table, bounce-back from the cell's own slot with the moving-wall and
pressure terms, the oracle's collision) must equal the oracle's step, for
Blocks along every axis and periodic or walled faces."""
import numpy as np
import pytest

Q = 19


def _classify(flags, periodic, face_bc, X, Y, Z):
    nz, ny, nx = flags.shape
    pos, n = [X, Y, Z], [nx, ny, nz]
    beyond, face = 0, 0
    for a in range(3):
        if 0 <= pos[a] < n[a]:
            continue
        if periodic[a]:
            pos[a] %= n[a]
        else:
            beyond += 1
            face = 2 * a + (0 if pos[a] < 0 else 1)
    if beyond >= 2:
        return 1, None
    if beyond == 1:
        return face_bc[face], None
    return int(flags[pos[2], pos[1], pos[0]]), tuple(pos)


def _list_layout(flags, bd, periodic, face_bc, e):
    nz, ny, nx = flags.shape
    nb = (nx // bd[0], ny // bd[1], nz // bd[2])
    index, cells = {}, []
    for bz in range(nb[2]):
        for by in range(nb[1]):
            for bx in range(nb[0]):
                for z in range(bd[2]):
                    for y in range(bd[1]):
                        for x in range(bd[0]):
                            X, Y, Z = bx * bd[0] + x, by * bd[1] + y, bz * bd[2] + z
                            if flags[Z, Y, X] == 0:
                                index[(X, Y, Z)] = len(cells)
                                cells.append((X, Y, Z))
    nbr = np.full((Q, len(cells)), -1, np.int64)
    for k, (X, Y, Z) in enumerate(cells):
        pres = 0
        for q in range(1, Q):
            kind, pos = _classify(flags, periodic, face_bc, X - e[q][0], Y - e[q][1], Z - e[q][2])
            if kind == 0:
                nbr[q, k] = index[pos]
            else:
                nbr[q, k] = {1: -1, 2: -2, 3: -3}[kind]
                pres |= kind == 3
        nbr[0, k] = pres
    return cells, nbr


@pytest.mark.parametrize("case", range(4))
def test_list_step_through_the_neighbour_table_equals_the_oracle(orc, case):
    rng = np.random.default_rng(60 + case)
    geoms = [((8, 6, 4), (4, 3, 2), (1, 0, 1), (1, 1, 2, 3, 1, 1)),
             ((8, 6, 4), (4, 3, 2), (0, 1, 0), (2, 3, 1, 1, 3, 2)),
             ((6, 6, 6), (3, 3, 3), (1, 1, 1), (1, 1, 1, 1, 1, 1)),
             ((9, 4, 6), (3, 4, 3), (0, 0, 1), (2, 3, 1, 1, 1, 1))]
    dims, bd, periodic, face_bc = geoms[case]
    flags = (rng.random(dims[::-1]) < 0.3).astype(np.uint8)
    flags[(flags != 0) & (rng.random(flags.shape) < 0.3)] = 2
    flags[(flags == 1) & (rng.random(flags.shape) < 0.3)] = 3
    wall_u, rho_b, rho0 = np.array([0.03, -0.01, 0.02]), 1.004, 1.0
    p = orc.Problem(dims=dims, tau=0.8, flags=flags, periodic=periodic, face_bc=face_bc,
                    collision=case % 2, wall_u=tuple(wall_u), rho_b=rho_b)
    e, w, opp = orc.lattice()
    e = e.astype(int)
    cells, nbr = _list_layout(flags, bd, periodic, face_bc, e)
    f = rng.uniform(-1e-2, 1e-2, (Q,) + dims[::-1]) * (flags == 0)
    S = np.array([[f[q, Z, Y, X] for (X, Y, Z) in cells] for q in range(Q)])  # the list arrays
    out = np.zeros_like(S)
    for k in range(len(cells)):
        g = np.empty(Q)
        g[0] = S[0, k]
        if nbr[0, k]:  # u_b of the pressure rule: the velocity of the cell's last collision
            ub = (e[1:].T @ S[1:, k]) / rho0
        for q in range(1, Q):
            s = nbr[q, k]
            if s >= 0:
                g[q] = S[q, s]
            else:
                v = S[opp[q], k]
                if s == -2:
                    v += 6 * w[q] * rho0 * (e[q] @ wall_u)
                elif s == -3:
                    eu = e[q] @ ub
                    v = -v + 2 * w[q] * ((rho_b - rho0) + rho0 * (4.5 * eu * eu - 1.5 * ub @ ub))
                g[q] = v
        out[:, k] = orc.collide(p, g)[0]
    ref = orc.step(p, f)
    want = np.array([[ref[q, Z, Y, X] for (X, Y, Z) in cells] for q in range(Q)])
    assert np.abs(out - want).max() < 1e-15
