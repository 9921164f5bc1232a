"""The oracle at the size of the headline workload (the 256^3-root molecular
cloud with three refinement levels, 2.76e7 cells): the walk over the full
tree against a closed form.

In the optically thin limit, an isotropic external field of energy E
falling on a convex box of surface S leaves E * 4 kappa_abs M / S in a
medium of mass M, whatever the density structure inside: the mean column
along the entering rays is 4 M / S (Cauchy's mean-chord theorem applied to
every volume element).  At 1 mm the cloud's mean optical depth is ~5e-7,
so the closed form holds to that order, and the Monte Carlo
estimate (continuous absorption: each package deposits along its whole
chord) scatters only with the chords' columns.  The same holds level by
level, since J = I in every cell.
"""
import numpy as np
import pytest

from paper_1206_3710_gb300 import synth


@pytest.fixture(scope="module")
def headline():
    return synth.cloud(n_root=256, levels=3, n_lambda=20, packets_per_bin=0, n_pix=16)


def test_headline_cloud_thin_limit(orc, headline):
    m = headline
    tree = orc.Tree(m.tree)
    level, leaf = tree.cells()
    assert tree.n_cells == m.tree.n_cells > 2.7e7 and int(level.max()) == 3
    o = m.optics
    b = int(np.argmax(o.lambda_um))
    one = synth.Optics(lambda_um=o.lambda_um[b:b + 1], kappa_ext=o.kappa_ext[b:b + 1], albedo=o.albedo[b:b + 1],
                       g_hg=o.g_hg[b:b + 1], dnu=o.dnu[b:b + 1])
    kabs = float((1 - o.albedo[b]) * o.kappa_ext[b])
    L = m.tree.box[0]
    h = L / m.tree.root[0] * 0.5 ** level
    M = float(np.sum(np.where(leaf, np.asarray(m.tree.density) * h ** 3, 0.0)))
    assert kabs * M / (L * L) < 1e-5   # optically thin
    E = 1.0
    src = synth.Source("external", bin_energy=np.array([E]))
    r = orc.trace(tree, [src], one, 20000, seed=11, n_threads=8)
    A = r["absorbed"][0]
    led = r["ledger"]
    assert np.all(A >= 0) and np.all(A[~leaf] == 0)
    assert abs(led["emitted"] - E) < 1e-12
    assert abs(led["emitted"] - led["absorbed"] - led["escaped"] - led["rr_loss"] + led["rr_gain"]) < 1e-12
    assert abs(A.sum() - led["absorbed"]) < 1e-9 * led["absorbed"]
    expect = 4 * kabs * M * E / (6 * L * L)
    assert abs(A.sum() / expect - 1) < 0.02
    # level by level (J = I in every cell, so each level takes its mass share);
    # the tolerance grows as the level's share of the crossings shrinks
    # (mass shares 0.60, 0.31, 0.094, 0.004)
    for lv, tol in ((0, 0.03), (1, 0.03), (2, 0.08), (3, 0.5)):
        s = leaf & (level == lv)
        m_l = float(np.sum(np.asarray(m.tree.density)[s] * h[s] ** 3))
        assert abs(A[s].sum() / (4 * kabs * m_l * E / (6 * L * L)) - 1) < tol, lv
