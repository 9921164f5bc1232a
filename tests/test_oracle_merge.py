"""Pins for the oracle's bottom-up construction of the hierarchical model
from a full-resolution cube (Sect. 4.1: combined cells have V-band optical
thickness <= 0.05 and density contrast < 30).

Checks against things the merge does not compute itself: closed forms for a
uniform cube, a single dense voxel, mass conservation, and a brute-force
walk over the tree that, for every leaf and every divided cell, slices the
full-resolution cells it covers straight out of the cube and tests the two
criteria (leaves satisfy them; a divided cell would violate one, or holds a
divided cell, which forbids combining it).
"""
import numpy as np
import pytest

from oracle.merge import merge_uniform


def _walk(desc, root):
    """(level, cx, cy, cz, refined, density) of every cell, from the level-ordered description."""
    n_ref, flags, dens = desc
    n0 = root[0] * root[1] * root[2]
    i = np.arange(n0)
    cells = [(0, int(k % root[0]), int((k // root[0]) % root[1]), int(k // (root[0] * root[1]))) for k in i]
    out = []
    pos = 0
    level_cells = cells
    lvl = 0
    while level_cells:
        nxt = []
        for (l, x, y, z) in level_cells:
            f = flags[pos]
            out.append((l, x, y, z, bool(f), dens[pos]))
            pos += 1
            if f:
                for o in range(8):
                    nxt.append((l + 1, 2 * x + (o & 1), 2 * y + ((o >> 1) & 1), 2 * z + ((o >> 2) & 1)))
        level_cells = nxt
        lvl += 1
    assert pos == flags.size
    return out


def _block(rho, L, l, x, y, z):
    s = 1 << (L - l)
    return rho[z * s:(z + 1) * s, y * s:(y + 1) * s, x * s:(x + 1) * s]


def test_uniform_cube_closed_form():
    root, L, box = (2, 3, 2), 3, (2.0, 3.0, 2.0)
    rho = np.full((2 << L, 3 << L, 2 << L), 2.5)
    # thin: everything combines into the root cells
    (n_ref, flags, dens), _ = merge_uniform(rho, root, box, kappa=0.01)
    assert flags.size == 12 and flags.sum() == 0 and np.all(dens == 2.5)
    # tau of a level-l cell = kappa rho 2^-l: 0.08, 0.04, ... -> stops at level 1
    (n_ref, flags, dens), _ = merge_uniform(rho, root, box, kappa=0.032)
    assert list(n_ref) == [12, 0] and flags.size == 12 + 96


def test_single_dense_voxel():
    root, L = (2, 2, 2), 3
    rho = np.ones((16, 16, 16))
    rho[5, 9, 3] = 100.0          # contrast 100 > 30 in every ancestor
    (n_ref, flags, dens), _ = merge_uniform(rho, root, (2.0,) * 3, kappa=1e-3)
    assert list(n_ref) == [1, 1, 1, 0]
    assert flags.size == 8 + 3 * 8
    cells = _walk((n_ref, flags, dens), root)
    deep = [c for c in cells if c[0] == L]
    assert sorted((c[1], c[2], c[3]) for c in deep if c[5] == 100.0) == [(3, 9, 5)]


@pytest.mark.parametrize("seed", [1, 2])
def test_criteria_by_brute_force_and_mass(seed):
    rng = np.random.default_rng(seed)
    root, L, box = (3, 2, 2), 3, (3.0, 2.0, 2.0)
    g = rng.normal(size=(2 << L, 2 << L, 3 << L))
    from scipy.ndimage import gaussian_filter
    rho = np.exp(1.5 * gaussian_filter(g, 1.5, mode="wrap") / gaussian_filter(g, 1.5, mode="wrap").std())
    kappa, tmax, cmax = 0.02, 0.05, 30.0
    desc, _ = merge_uniform(rho, root, box, kappa, tmax, cmax)
    n_ref, flags, dens = desc
    cells = _walk(desc, root)
    h0 = box[0] / root[0]
    mass = 0.0
    n_leaf_levels = set()
    for (l, x, y, z, refined, d) in cells:
        blk = _block(rho, L, l, x, y, z)
        h = h0 * 0.5 ** l
        tau_ok = kappa * blk.mean() * h <= tmax * (1 + 1e-12)
        c_ok = blk.max() < cmax * blk.min()
        if not refined:
            n_leaf_levels.add(l)
            assert l == L or (tau_ok and c_ok), (l, x, y, z)
            np.testing.assert_allclose(d, blk.mean(), rtol=1e-12)
            mass += d * h ** 3
        elif l < L:
            kids = [c for c in cells if c[0] == l + 1 and (c[1] >> 1, c[2] >> 1, c[3] >> 1) == (x, y, z)]
            assert len(kids) == 8
            assert (not tau_ok) or (not c_ok) or any(k[4] for k in kids), (l, x, y, z)
    np.testing.assert_allclose(mass, rho.sum() * (h0 * 0.5 ** L) ** 3, rtol=1e-12)
    assert len(n_leaf_levels) >= 3  # the field is refined where it is dense or contrasted
