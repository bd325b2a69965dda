"""Pins of the oracle's geometry and random-number generator.

Site numbering, coordinates and colour follow Sec. 2, eqs. (i_s), (xD),
(x^i), (i_c); the DLT neighbour rule follows Sec. 2.2.  They are checked here
against numpy's Fortran-order index routines and brute-force enumeration.
"""
import itertools
import os

import numpy as np
import pytest

import oracle

SHAPES = [[4, 4], [2, 4, 6], [4, 2, 2, 4], [2, 2, 4, 2, 2]]


@pytest.mark.parametrize("dims", SHAPES)
def test_site_number_round_trip(dims):
    lat = oracle.Lattice(dims)
    V = int(np.prod(dims))
    for s in range(V):
        x = lat.site_coords(s)
        # eq. (i_s) with x^1 fastest is Fortran (column-major) order.
        assert s == int(np.ravel_multi_index(tuple(x), dims, order="F"))
        assert lat.site_index(x) == s
        assert lat.colour(x) == sum(x) % 2


@pytest.mark.parametrize("dims", SHAPES)
def test_pbc_neighbours_brute_force(dims):
    lat = oracle.Lattice(dims)
    tab = lat.neighbour_table()
    D = len(dims)
    for x in itertools.product(*[range(n) for n in dims]):
        s = int(np.ravel_multi_index(x, dims, order="F"))
        for mu in range(D):
            for d, step in ((0, -1), (1, +1)):
                y = list(x)
                y[mu] = (y[mu] + step) % dims[mu]
                assert tab[0, s, mu, d] == int(np.ravel_multi_index(tuple(y), dims, order="F"))
                # one step in any direction flips the checkerboard colour (even extents)
                assert lat.colour(y) != lat.colour(list(x))


@pytest.mark.parametrize("glue_mask", [0b1111, 0b1000, 0b0111, 0b0101])
def test_dlt_neighbours(glue_mask):
    dims = [4, 2, 2, 4]
    lat = oracle.Lattice(dims, nlayers=2, glue_mask=glue_mask)
    tab = lat.neighbour_table()
    V = lat.V
    for layer in range(2):
        for x in itertools.product(*[range(n) for n in dims]):
            s = int(np.ravel_multi_index(x, dims, order="F"))
            for mu in range(4):
                for d, step in ((0, -1), (1, +1)):
                    y = list(x)
                    y[mu] += step
                    crossed = y[mu] < 0 or y[mu] >= dims[mu]
                    y[mu] %= dims[mu]
                    l2 = 1 - layer if (crossed and (glue_mask >> mu) & 1) else layer
                    want = l2 * V + int(np.ravel_multi_index(tuple(y), dims, order="F"))
                    assert tab[layer, s, mu, d] == want


def test_dlt_plaquettes_close():
    """x + mu - nu is the same site whichever step is taken first, so every
    plaquette of the DLT is a closed loop (Sec. 2.2)."""
    dims = [4, 4, 2, 2]
    lat = oracle.Lattice(dims, nlayers=2, glue_mask=0b1011)
    tab = lat.neighbour_table().reshape(2 * lat.V, 4, 2)
    for site in range(2 * lat.V):
        for mu in range(4):
            for nu in range(4):
                if nu == mu:
                    continue
                a = tab[tab[site, mu, 1], nu, 0]
                b = tab[tab[site, nu, 0], mu, 1]
                assert a == b


def test_dlt_two_dimensional_self_loop():
    """On a 2-D DLT glued in both directions the shortest closed line through
    the boundary runs along the diagonal (Sec. 2.2): two steps across the
    boundary are needed to come back to the same layer."""
    n = 4
    lat = oracle.Lattice([n, n], nlayers=2, glue_mask=0b11)
    tab = lat.neighbour_table().reshape(2 * lat.V, 2, 2)
    site = 0
    for _ in range(n):  # n steps in direction 1 cross the boundary once
        site = tab[site, 0, 1]
    assert site == lat.V  # same coordinates, other layer
    for _ in range(n):
        site = tab[site, 0, 1]
    assert site == 0


def _kat():
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert oracle.philox4x32_10(ctr, key) == out
