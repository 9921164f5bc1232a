"""Pins for package splitting and roulette at grid boundaries (Sect. 2.3,
Table 1), in the oracle.

A package that enters a grid dl levels deeper becomes N^dl packages of
weight W/N^dl; one that leaves for a grid dl levels shallower survives with
probability N^-dl and carries N^dl W.  Checks: along a straight line through
a pure absorber the copies deposit exactly what the unsplit package would
inside the refined region; the count of copies; exact energy bookkeeping;
the binomial statistics of the exit roulette; unchanged expectations with
scattering; and the noise reduction at the deepest level for an external
field (Table 1).
"""
import math

import numpy as np
import pytest

from paper_1206_3710_gb300 import synth


def _optics(kext, albedo=0.0, g=0.0):
    return synth.Optics(lambda_um=np.array([0.55]), kappa_ext=np.array([kext]), albedo=np.array([albedo]),
                        g_hg=np.array([g]), dnu=np.ones(1))


class _Beam:
    kind = "beam"

    def __init__(self, pos, dir_, energy=1.0):
        self.pos, self.dir, self.bin_energy = pos, dir_, np.array([energy])


def _block_tree(rho=1.0):
    """4^3 root cells of side 1; the root cells with x index 1 or 2 refined once."""
    return synth.grow_tree((4, 4, 4), (4.0,) * 3, 1, lambda l, x, y, z: np.full(x.size, rho),
                           lambda l, x, y, z, r: (x == 1) | (x == 2))


def _nested_tree(levels=3, contrast=1.0):
    """4^3 root cells of side 1 and a nest refined towards the centre of the
    box (levels 1 and 3 hold leaves); the density of level l is contrast^l."""
    def refine(l, x, y, z, r):
        c = 2 * 2 ** l  # centre of the box in cells of level l
        h = 0.75 * 2 ** l
        return (np.abs(x + 0.5 - c) < h) & (np.abs(y + 0.5 - c) < h) & (np.abs(z + 0.5 - c) < h)
    return synth.grow_tree((4, 4, 4), (4.0,) * 3, levels, lambda l, x, y, z: np.full(x.size, contrast ** l), refine)


def test_split_beam_pure_absorber_exact(orc):
    tree = orc.Tree(_block_tree())
    level, leaf = tree.cells()
    tau_per_cell = 0.3
    o = _optics(tau_per_cell)
    n = 500
    beam = _Beam((0.0, 1.3, 2.7), (1.0, 0.0, 0.0))
    plain = orc.trace(tree, [beam], o, n, seed=4)
    split = orc.trace(tree, [beam], o, n, seed=4, split_factor=4)
    A0, A1 = plain["absorbed"][0], split["absorbed"][0]
    # every package enters the refined block once: three copies each
    assert split["ledger"]["n_split"] == 3 * n
    # before the block and inside it the four quarters deposit what one package would
    inside = leaf & (level == 1)
    # the beam crosses two root cells: the first (largest deposit) and the one after the block
    before = leaf & (level == 0) & (A0 == A0[leaf & (level == 0)].max())
    np.testing.assert_allclose(A1[inside], A0[inside], rtol=1e-12, atol=0)
    np.testing.assert_allclose(A1[before], A0[before], rtol=1e-12)
    # exact bookkeeping, the exit roulette booked as roulette gain and loss
    L = split["ledger"]
    assert abs(L["emitted"] - L["absorbed"] - L["escaped"] - L["rr_loss"] + L["rr_gain"]) < 1e-12
    assert L["rr_loss"] > 0 and L["rr_gain"] > 0
    # after the block: K ~ Bin(4, 1/4) survivors per package, each carrying W
    after_cell = leaf & (level == 0) & (A0 > 0) & ~before
    assert after_cell.sum() == 1
    f = A0[after_cell][0] / n  # one package's deposit there
    K = A1[after_cell][0] / f
    assert abs(K - round(K)) < 1e-9  # a whole number of survivors
    sig = math.sqrt(n * 4 * 0.25 * 0.75)
    assert abs(K - n) < 4 * sig
    np.testing.assert_allclose(split["ledger"]["escaped"] / plain["ledger"]["escaped"], K / n, rtol=1e-12)


def test_split_factor_one_is_plain(orc):
    tree = orc.Tree(_nested_tree())
    o = _optics(0.8, albedo=0.6, g=0.3)
    ext = synth.Source("external", bin_energy=np.array([1.0]))
    a = orc.trace(tree, [ext], o, 3000, seed=9)
    b = orc.trace(tree, [ext], o, 3000, seed=9, split_factor=1)
    np.testing.assert_array_equal(a["absorbed"], b["absorbed"])
    assert b["ledger"]["n_split"] == 0


def test_split_limits(orc):
    tree = orc.Tree(_nested_tree(levels=3))
    o = _optics(0.8, albedo=0.6)
    ext = synth.Source("external", bin_energy=np.array([1.0]))
    with pytest.raises(RuntimeError):
        orc.trace(tree, [ext], o, 10, seed=1, split_factor=8)  # 8^3 = 512 > 256 packages per split
    r = orc.trace(tree, [ext], o, 200, seed=1, split_factor=8, split_max_level=2)
    assert r["ledger"]["n_split"] > 0


def _level_sums(tree, A):
    level, leaf = tree.cells()
    return np.array([A[leaf & (level == l)].sum() for l in range(level.max() + 1)])


@pytest.mark.parametrize("kind", ["external", "point"])
def test_split_same_expectation(orc, kind):
    """With scattering, the absorbed energy summed over each level agrees
    with the unsplit run (independent seeds, 4 sigma of the run-to-run
    scatter), and energy is conserved in every run."""
    tree = orc.Tree(_nested_tree())
    o = _optics(1.2, albedo=0.5, g=0.4)
    src = synth.Source("external", bin_energy=np.array([1.0])) if kind == "external" else \
        synth.Source("point", bin_energy=np.array([1.0]), pos=(2.03, 1.96, 2.11))
    runs = {1: [], 2: []}
    for N in runs:
        for s in range(8):
            r = orc.trace(tree, [src], o, 4000, seed=100 + s, split_factor=N, rr_wmin=1e-3, rr_p=0.5,
                          n_threads=4)
            L = r["ledger"]
            assert abs(L["emitted"] - L["absorbed"] - L["escaped"] - L["rr_loss"] + L["rr_gain"]) < 1e-10
            runs[N].append(_level_sums(tree, r["absorbed"][0]))
    a, b = np.array(runs[1]), np.array(runs[2])
    sig = np.sqrt(a.var(axis=0, ddof=1) / len(a) + b.var(axis=0, ddof=1) / len(b))
    assert np.all(np.abs(a.mean(axis=0) - b.mean(axis=0)) < 4 * sig + 1e-15)


def test_split_reduces_deep_noise_external(orc):
    """Table 1, external radiation: with the same number of packages sent,
    splitting lowers the cell-by-cell noise (RMS about the mean of the runs,
    Sect. 4.1) of the deepest level, a dense core, while the root level keeps
    its noise.  Copies leave the entry point along the same line, so the
    gain comes from their independent scatterings inside the core."""
    tree = orc.Tree(_nested_tree(contrast=4.0))
    level, leaf = tree.cells()
    o = _optics(1.0, albedo=0.5, g=0.3)
    ext = synth.Source("external", bin_energy=np.array([1.0]))
    noise = {}
    for N in (1, 4):
        A = np.array([orc.trace(tree, [ext], o, 3000, seed=200 + s, split_factor=N, n_threads=4)["absorbed"][0]
                      for s in range(12)])
        ref = A.mean(axis=0)
        noise[N] = {l: np.sqrt(np.mean((A[:, leaf & (level == l)] - ref[leaf & (level == l)]) ** 2)) /
                    np.mean(ref[leaf & (level == l)]) for l in (0, 1, 3)}
    assert noise[4][3] < 0.8 * noise[1][3]
    assert abs(noise[4][0] / noise[1][0] - 1.0) < 0.1
