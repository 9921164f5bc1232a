"""Pins for the oracle's importance-sampled dust emission: the emission cell
of a dust package drawn by weights other than the emission, each package
carrying emission_c / (N p_c), so that every cell still emits its energy in
expectation (the standard importance-sampling estimator).  Checks: weights
proportional to the emission reproduce the plain draw; any positive weights
leave the expected absorbed field and each cell's emitted energy unchanged;
a cell that emits but can never be drawn is rejected."""
import numpy as np
import pytest

from paper_1206_3710_gb300 import synth


def _model():
    L = 20 * synth.AU_CM
    desc = synth.random_refined_tree((6, 6, 6), (L,) * 3, 2, 0.35, 21,
                                     rho_fn=lambda l, x, y, z: np.random.default_rng(l + 3).uniform(0.5e-18, 2e-18,
                                                                                                    x.size))
    lam = synth.log_lambda_grid(4)
    optics = synth.powerlaw_dust(lam, 2.0 / (1e-18 * L), 1.0)
    return desc, optics


def _emission(orc, tree, optics, seed=2):
    level, leaf = tree.cells()
    T = np.where(leaf, np.random.default_rng(seed).uniform(60.0, 400.0, tree.n_cells), 0.0)
    kabs = (1 - optics.albedo) * optics.kappa_ext
    return orc.dust_emission(tree, T, optics.lambda_um, kabs, optics.dnu)


def test_sampling_proportional_to_emission_is_the_plain_draw(orc):
    desc, optics = _model()
    tree = orc.Tree(desc)
    em = _emission(orc, tree, optics)
    a = orc.trace(tree, [orc._DustSource(em)], optics, 3000, seed=4, iter_=1, rr_wmin=1e-3, rr_p=0.5)
    b = orc.trace(tree, [orc._DustSource(em, sampling=4.0 * em)], optics, 3000, seed=4, iter_=1, rr_wmin=1e-3,
                  rr_p=0.5)
    np.testing.assert_allclose(b["absorbed"], a["absorbed"], rtol=1e-12, atol=1e-14 * a["absorbed"].max())
    for k in ("emitted", "absorbed", "escaped"):
        assert b["ledger"][k] == pytest.approx(a["ledger"][k], rel=1e-12)
    assert b["ledger"]["n_cross"] == a["ledger"]["n_cross"]


def test_sampling_keeps_expectations(orc):
    """Cells drawn by the emission times a random factor in [0.05, 20]: the
    emitted energy per cell (self-emission tally) and the absorbed energy per
    level agree with the plain draw within 4 sigma of the run-to-run scatter,
    and the ledger closes in every run."""
    desc, optics = _model()
    tree = orc.Tree(desc)
    level, leaf = tree.cells()
    em = _emission(orc, tree, optics)
    f = np.exp(np.random.default_rng(7).uniform(np.log(0.05), np.log(20.0), em.shape))
    nl = len(optics.kappa_ext)
    runs = {False: [], True: []}
    emit = {False: [], True: []}
    for imp in runs:
        for s in range(10):
            se = np.zeros((nl, tree.n_cells))
            src = orc._DustSource(em, sampling=em * f if imp else None)
            r = orc.trace(tree, [src], optics, 2000, seed=30 + s, iter_=1, rr_wmin=1e-3, rr_p=0.5, n_threads=4,
                          self_emitted=se)
            L = r["ledger"]
            assert abs(L["emitted"] - L["absorbed"] - L["escaped"] - L["rr_loss"] + L["rr_gain"]) < 1e-10 * L["emitted"]
            A = r["absorbed"].sum(axis=0)
            runs[imp].append([A[leaf & (level == l)].sum() for l in range(level.max() + 1)])
            emit[imp].append(se.sum(axis=0)[leaf])
    a, b = np.array(runs[False]), np.array(runs[True])
    sig = np.sqrt(a.var(axis=0, ddof=1) / len(a) + b.var(axis=0, ddof=1) / len(b))
    assert np.all(np.abs(a.mean(axis=0) - b.mean(axis=0)) < 4 * sig)
    # emitted energy against the exact emission, in 40 random groups of leaves
    # (a single cell is drawn too rarely for a per-cell test)
    e_exact = em.sum(axis=0)[leaf]
    grp = np.random.default_rng(8).integers(0, 40, e_exact.size)
    for imp in emit:
        g = np.array([np.bincount(grp, weights=e, minlength=40) for e in emit[imp]])
        ge = np.bincount(grp, weights=e_exact, minlength=40)
        s_g = g.std(axis=0, ddof=1) / np.sqrt(len(g))
        assert np.all(np.abs(g.mean(axis=0) - ge) < 4 * s_g + 1e-9 * ge)


def test_sampling_must_cover_the_emission(orc):
    desc, optics = _model()
    tree = orc.Tree(desc)
    em = _emission(orc, tree, optics)
    samp = em.copy()
    c = int(np.argmax(em[0]))
    samp[0, c] = 0.0
    with pytest.raises(RuntimeError):
        orc.trace(tree, [orc._DustSource(em, sampling=samp)], optics, 100, seed=1, iter_=1)
