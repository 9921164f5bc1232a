"""Pins for the oracle's tree and cell stepping (Sects. 2.1 and 2.3).

The reference for a walk is brute force: every leaf's axis-aligned box is
rebuilt from the level-ordered layout, each is intersected with the ray by
the slab method, and the leaves are sorted by entry distance.
"""
import numpy as np
import pytest

from paper_1206_3710_gb300 import synth


def leaf_boxes(desc):
    """(id, lo[3], size) in root-cell units of every leaf, from the layout."""
    rx, ry, rz = desc.root
    cz, cy, cx = np.meshgrid(np.arange(rz), np.arange(ry), np.arange(rx), indexing="ij")
    coords = [(cx.ravel(), cy.ravel(), cz.ravel())]
    off = desc.level_offsets()
    out = []
    for lev in range(desc.n_levels):
        x, y, z = coords[-1]
        flags = desc.refine_flags[off[lev]:off[lev + 1]].astype(bool)
        size = 0.5 ** lev
        for i in np.nonzero(~flags)[0]:
            out.append((off[lev] + i, np.array([x[i], y[i], z[i]]) * size, size))
        o = np.arange(8)
        coords.append(((2 * x[flags][:, None] + (o & 1)).ravel(),
                       (2 * y[flags][:, None] + ((o >> 1) & 1)).ravel(),
                       (2 * z[flags][:, None] + ((o >> 2) & 1)).ravel()))
    return out


def brute_walk(boxes, o, d):
    segs = []
    for cid, lo, size in boxes:
        t0, t1 = -np.inf, np.inf
        for a in range(3):
            if d[a] == 0:
                if not (lo[a] <= o[a] < lo[a] + size):
                    t0, t1 = 1, 0
                continue
            ta = (lo[a] - o[a]) / d[a]
            tb = (lo[a] + size - o[a]) / d[a]
            t0 = max(t0, min(ta, tb))
            t1 = min(t1, max(ta, tb))
        t0 = max(t0, 0.0)
        if t1 > t0:
            segs.append((t0, cid, t1 - t0))
    segs.sort()
    return [s[1] for s in segs], np.array([s[2] for s in segs])


@pytest.mark.parametrize("seed", range(6))
def test_walk_matches_brute_force(orc, seed):
    desc = synth.random_refined_tree((3, 4, 2), (3.0, 4.0, 2.0), 2, 0.45, seed)
    tree = orc.Tree(desc)
    boxes = leaf_boxes(desc)
    assert len(boxes) == int((desc.refine_flags == 0).sum())
    rng = np.random.default_rng(100 + seed)
    h0 = desc.box[0] / desc.root[0]
    n_checked = 0
    for _ in range(150):
        o = rng.uniform(0, 1, 3) * np.array(desc.root)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        cells, lens, marg = orc.walk(tree, o * h0, d)
        bc, bl = brute_walk(boxes, o, d)
        assert list(cells) == bc
        np.testing.assert_allclose(lens / h0, bl, rtol=1e-12, atol=1e-13)
        n_checked += 1
    assert n_checked == 150


def test_walk_axis_aligned_and_face_ties(orc):
    """Rays on cell faces: a point on a face belongs to the cell the ray moves
    into, and a ray lying in a face plane uses the upper cell (half-open)."""
    desc = synth.uniform_tree((4, 4, 4), (4.0, 4.0, 4.0), 1.0)
    tree = orc.Tree(desc)
    cells, lens, _ = orc.walk(tree, [0.0, 2.0, 2.0], [1.0, 0.0, 0.0])
    # y = z = 2 exactly: upper cells iy = iz = 2
    assert list(cells) == [0 + 4 * (2 + 4 * 2) + i for i in range(4)]
    np.testing.assert_array_equal(lens, np.ones(4))
    cells, lens, _ = orc.walk(tree, [4.0, 1.5, 1.5], [-1.0, 0.0, 0.0])
    assert list(cells) == [i + 4 * (1 + 4 * 1) for i in (3, 2, 1, 0)]
    # starting on an interior face moving down: first cell is the lower one
    cells, _, _ = orc.walk(tree, [2.0, 0.5, 0.5], [-1.0, 0.0, 0.0])
    assert list(cells) == [1, 0]


def test_tree_rejects_inconsistent(orc):
    desc = synth.random_refined_tree((2, 2, 2), (2.0, 2.0, 2.0), 2, 0.5, 3)
    bad = synth.TreeDesc(desc.root, desc.box, desc.n_refined + np.array([1] + [0] * (desc.n_levels - 1)),
                         desc.refine_flags, desc.density)
    with pytest.raises(ValueError):
        orc.Tree(bad)
    dens = desc.density.copy()
    leaf = np.nonzero(desc.refine_flags == 0)[0][0]
    dens[leaf] = -1.0
    with pytest.raises(ValueError):
        orc.Tree(synth.TreeDesc(desc.root, desc.box, desc.n_refined, desc.refine_flags, dens))
    with pytest.raises(ValueError):   # non-cubic cells
        orc.Tree(synth.TreeDesc(desc.root, (2.0, 2.0, 3.0), desc.n_refined, desc.refine_flags, desc.density))


def test_tree_cells(orc):
    desc = synth.random_refined_tree((3, 2, 2), (3.0, 2.0, 2.0), 3, 0.4, 11)
    tree = orc.Tree(desc)
    lev, leaf = tree.cells()
    assert tree.n_cells == desc.n_cells
    np.testing.assert_array_equal(lev, desc.cell_levels())
    np.testing.assert_array_equal(leaf, desc.refine_flags == 0)


def test_walk_lengths_sum_to_chord(orc):
    """Total path length equals the analytic chord of the root box."""
    desc = synth.random_refined_tree((4, 4, 4), (4.0, 4.0, 4.0), 2, 0.3, 2)
    tree = orc.Tree(desc)
    rng = np.random.default_rng(7)
    for _ in range(100):
        o = rng.uniform(0, 4, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        t_exit = min(((4.0 if d[a] > 0 else 0.0) - o[a]) / d[a] for a in range(3))
        _, lens, _ = orc.walk(tree, o, d)
        assert abs(lens.sum() - t_exit) < 1e-12 * 4
