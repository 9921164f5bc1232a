"""Pins for the oracle's dust packages (Sect. 4.2: the number of packages a
cell sends at a frequency follows its emission there, every package of the
frequency carrying the same energy w_b).  Cell c sends floor(E_bc / w_b +
u_bc) packages, u_bc fixed by the run's key, and package j of cell c draws
from the cell's own stream.  Checks: each count is within one of E_bc / w_b
and their average over keys is E_bc / w_b; the emitted energy is the
packages' energy; a change in one cell's emission changes only that cell's
packages (so repeated runs keep their random numbers, the point of the
common streams of the Lambda iteration); the cells of a subtree send exactly
the packages they send in the whole model (subiterations, App. B); and the
Lambda iteration of a small disc, which with packages drawn one by one from
the cumulative emission stalled at max dT/T ~ 0.2, meets the 1e-3 stop rule."""
import math

import numpy as np
import pytest

from paper_1206_3710_gb300 import synth


def _model(n_lambda=1):
    L = 20 * synth.AU_CM
    desc = synth.random_refined_tree((6, 6, 6), (L,) * 3, 2, 0.35, 21,
                                     rho_fn=lambda l, x, y, z: np.random.default_rng(l + 3).uniform(0.5e-18, 2e-18,
                                                                                                    x.size))
    lam = synth.log_lambda_grid(n_lambda) if n_lambda > 1 else np.array([30.0])
    optics = synth.powerlaw_dust(lam, 2.0 / (1e-18 * L), 1.0)
    return desc, optics


def _emission(orc, tree, optics, seed=2):
    level, leaf = tree.cells()
    T = np.where(leaf, np.random.default_rng(seed).uniform(60.0, 400.0, tree.n_cells), 0.0)
    kabs = (1 - optics.albedo) * optics.kappa_ext
    return orc.dust_emission(tree, T, optics.lambda_um, kabs, optics.dnu)


def _counts(orc, tree, optics, em, npk, seed, w=None):
    """packages per cell (the self-emission count tally), ledger, absorbed"""
    nl, nc = em.shape
    sa, se, sn = np.zeros((nl, nc)), np.zeros((nl, nc)), np.zeros(nc)
    r = orc.trace(tree, [orc._DustSource(em, package_energy=w)], optics, npk, seed=seed, iter_=1,
                  self_absorbed=sa, self_emitted=se, self_count=sn, n_threads=4)
    return sn, r


def test_counts_within_one_of_the_emission(orc):
    desc, optics = _model()
    tree = orc.Tree(desc)
    em = _emission(orc, tree, optics)
    npk = 5000
    n, r = _counts(orc, tree, optics, em, npk, seed=4)
    w = em.sum() / npk
    x = em[0] / w
    assert np.all(n >= np.floor(x)) and np.all(n <= np.ceil(x))
    assert n.sum() == r["ledger"]["n_packets"]
    assert abs(n.sum() - npk) < 4 * math.sqrt(len(x))            # rounding noise only
    assert r["ledger"]["emitted"] == pytest.approx(n.sum() * w, rel=1e-12)
    L = r["ledger"]
    assert abs(L["emitted"] - L["absorbed"] - L["escaped"]) < 1e-10 * L["emitted"]


def test_counts_average_to_the_emission(orc):
    """Over 300 keys the mean count of each cell is E_c / w (the rounding
    uniform makes floor(x + u) an unbiased count)."""
    desc, optics = _model()
    tree = orc.Tree(desc)
    em = _emission(orc, tree, optics)
    npk = 600
    w = em.sum() / npk
    x = em[0] / w
    S = 300
    tot = np.zeros_like(x)
    for s in range(S):
        n, _ = _counts(orc, tree, optics, em, npk, seed=100 + s)
        tot += n
    frac = x - np.floor(x)
    sd = np.sqrt(np.maximum(frac * (1 - frac), 1e-12) / S)
    z = (tot / S - x) / sd
    ok = frac > 0.02
    assert np.mean(np.abs(z[ok]) > 3) < 0.01
    assert abs(z[ok].mean()) < 4 / math.sqrt(ok.sum())


def test_one_cells_change_moves_only_its_packages(orc):
    """Raising one cell's emission adds packages of that cell and leaves
    every other package as it was: the absorbed fields differ by exactly what
    that cell's packages deposit (package energy held fixed)."""
    desc, optics = _model()
    tree = orc.Tree(desc)
    level, leaf = tree.cells()
    em = _emission(orc, tree, optics)
    npk = 4000
    w = np.array([em.sum() / npk])
    k = int(np.argmax(em[0]))
    em2 = em.copy()
    em2[0, k] *= 1.7
    only1 = np.zeros_like(em)
    only1[0, k] = em[0, k]
    only2 = np.zeros_like(em)
    only2[0, k] = em2[0, k]
    a = _counts(orc, tree, optics, em, npk, 9, w)[1]["absorbed"]
    b = _counts(orc, tree, optics, em2, npk, 9, w)[1]["absorbed"]
    a1 = _counts(orc, tree, optics, only1, npk, 9, w)[1]["absorbed"]
    b1 = _counts(orc, tree, optics, only2, npk, 9, w)[1]["absorbed"]
    np.testing.assert_allclose(b - a, b1 - a1, rtol=0, atol=1e-10 * np.abs(a).max())
    assert np.abs(b1 - a1).max() > 1e-3 * np.abs(a).max()


def test_subtree_sends_its_packages_of_the_whole_model(orc):
    """With the whole model's package energy, the cells of a subset send the
    packages they send in the whole model: the two halves' absorbed fields
    add up to the whole's."""
    desc, optics = _model(n_lambda=3)
    tree = orc.Tree(desc)
    level, leaf = tree.cells()
    em = _emission(orc, tree, optics)
    npk = np.array([3000, 2000, 1000])
    w = em.sum(axis=1) / npk
    deep = (level >= 1)[None, :]
    whole = _counts(orc, tree, optics, em, npk, 12, w)[1]
    part_d = _counts(orc, tree, optics, em * deep, npk, 12, w)[1]
    part_s = _counts(orc, tree, optics, em * ~deep, npk, 12, w)[1]
    np.testing.assert_allclose(part_d["absorbed"] + part_s["absorbed"], whole["absorbed"], rtol=1e-10,
                               atol=1e-12 * whole["absorbed"].max())
    assert part_d["ledger"]["n_packets"] + part_s["ledger"]["n_packets"] == whole["ledger"]["n_packets"]


def test_disc_lambda_iteration_meets_the_stop_rule(orc):
    """Sect. 4.2's disc, small: 27,200 cells, 12 wavelengths.  With the
    packages tied to their cells the iteration's common random numbers hold
    from step to step, so max dT/T over cells with >= 1e3 deposits falls
    below 1e-3 (drawing each package's cell from the cumulative emission
    moved a third of them to other cells each step, and the change stalled
    near 0.2)."""
    m = synth.disc(n_root=16, max_level=6, n_lambda=12, packets=0, target_cells=3e4, max_cells=200000)
    tree = orc.Tree(m.tree)
    T, hist = orc.lambda_iterate(tree, m.sources[0], m.optics, 30000, 30000, seed=3, tol=1e-3, max_iter=30,
                                 min_hits=1000, n_threads=8)
    assert hist[-1] < 1e-3, hist
    assert len(hist) < 30
