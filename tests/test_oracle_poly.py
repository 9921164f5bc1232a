"""Pins for polychromatic packages (Sect. 2.3, after Jonsson 2006) in the
oracle: a package carries one weight per bin of its group, its path is
drawn at the group's reference bin and each weight carries the likelihood
ratio of that path.

Checks against things the polychromatic path does not compute itself: the
closed-form transmission of a pure absorber per bin; the reference bin
(for groups of two, the first bin, whose random stream is the
monochromatic package's) reproducing the monochromatic run exactly; and the
other bins agreeing with monochromatic runs in expectation.
"""
import math

import numpy as np
import pytest

from paper_1206_3710_gb300 import synth


class _Beam:
    kind = "beam"

    def __init__(self, pos, dir_, energy):
        self.pos, self.dir, self.bin_energy = pos, dir_, np.asarray(energy, dtype=float)


def _optics(kext, albedo, g):
    n = len(kext)
    return synth.Optics(lambda_um=np.linspace(0.5, 1.0, n), kappa_ext=np.asarray(kext, float),
                        albedo=np.asarray(albedo, float), g_hg=np.asarray(g, float), dnu=np.ones(n))


def _tree(seed=3):
    return synth.random_refined_tree((4, 4, 4), (4.0,) * 3, 2, 0.3, seed,
                                     rho_fn=lambda l, x, y, z: np.random.default_rng(l + 7).uniform(0.5, 1.5, x.size))


def test_poly_pure_absorber_closed_form(orc):
    """Albedo 0 in every bin: no scattering, so each bin's absorbed total is
    N W0_j (1 - e^{-tau_j}) along the beam through a uniform cube."""
    L, rho = 4.0, 1.0
    tree = orc.Tree(synth.uniform_tree((4, 4, 4), (L,) * 3, rho))
    kext = np.array([0.1, 0.3, 0.05, 0.6])
    E = np.array([1.0, 2.0, 0.5, 1.5])
    o = _optics(kext, [0, 0, 0, 0], [0, 0, 0, 0])
    n = 300
    r = orc.trace(tree, [_Beam((0.0, 1.3, 2.7), (1.0, 0.0, 0.0), E)], o, n, seed=5, poly_group=4)
    tot = r["absorbed"].sum(axis=1)
    np.testing.assert_allclose(tot, E * (1 - np.exp(-kext * rho * L)), rtol=1e-12)
    assert r["ledger"]["n_packets"] == n


def test_poly_reference_bin_is_the_monochromatic_package(orc):
    """Groups of two: the reference is the first bin, whose stream is that of
    the monochromatic package of the bin; its absorbed energy, images and the
    packages' scattering counts equal the monochromatic run's."""
    tree = orc.Tree(_tree())
    o = _optics([0.9, 0.5, 1.4, 0.3], [0.6, 0.3, 0.7, 0.5], [0.3, 0.6, 0.1, 0.4])
    src = synth.Source("external", bin_energy=np.array([1.0, 0.7, 1.3, 0.4]))
    obs = synth.axis_observers(12, 4.0, "all6")
    kw = dict(seed=11, observers=obs, rr_wmin=1e-3, rr_p=0.5, record=True)
    mono = orc.trace(tree, [src], o, 800, **kw)
    poly = orc.trace(tree, [src], o, 800, poly_group=2, **kw)
    for b in (0, 2):
        np.testing.assert_allclose(poly["absorbed"][b], mono["absorbed"][b], rtol=1e-11,
                                   atol=1e-14 * mono["absorbed"][b].max())
        np.testing.assert_allclose(poly["images"][:, b], mono["images"][:, b], rtol=1e-11,
                                   atol=1e-14 * mono["images"][:, b].max())
    # the packages of group 0 are the monochromatic packages of bin 0: same
    # scatterings and fates
    rp, rm = poly["rec"], mono["rec"]
    n0 = 800
    assert np.array_equal(rp[:n0, 1], rm[:n0, 1]) and np.array_equal(rp[:n0, 3], rm[:n0, 3])
    assert poly["ledger"]["n_packets"] == 2 * n0


@pytest.mark.parametrize("kind", ["external", "point"])
def test_poly_expectation_matches_monochromatic(orc, kind):
    """Every bin of a group of four, including the reweighted ones, agrees
    with monochromatic runs in its absorbed energy per level and its escaped
    light (independent seeds, 4 sigma of the run-to-run scatter)."""
    desc = _tree(5)
    tree = orc.Tree(desc)
    level, leaf = tree.cells()
    o = _optics([0.8, 1.0, 1.3, 0.6], [0.5, 0.6, 0.55, 0.4], [0.3, 0.4, 0.2, 0.35])
    E = np.array([1.0, 0.8, 1.2, 0.6])
    src = synth.Source("external", bin_energy=E) if kind == "external" else \
        synth.Source("point", bin_energy=E, pos=(2.03, 1.96, 2.11))
    obs = synth.axis_observers(4, 4.0, "all6")
    stats = {}
    for F in (1, 4):
        vals = []
        for s in range(8):
            r = orc.trace(tree, [src], o, 3000, seed=300 + s, poly_group=F, observers=obs, n_threads=4)
            A = r["absorbed"]
            v = [A[b, leaf & (level == l)].sum() for b in range(4) for l in range(3)]
            v += list(r["images"].sum(axis=(0, 2, 3)))
            vals.append(v)
        stats[F] = np.array(vals)
    a, b = stats[1], stats[4]
    sig = np.sqrt(a.var(axis=0, ddof=1) / len(a) + b.var(axis=0, ddof=1) / len(b))
    assert np.all(np.abs(a.mean(axis=0) - b.mean(axis=0)) < 4 * sig + 1e-15)


def test_poly_rejects_unsupported(orc):
    tree = orc.Tree(_tree())
    o = _optics([0.9, 0.5], [0.0, 0.3], [0.3, 0.6])  # reference bin 0 does not scatter, bin 1 does
    src = synth.Source("external", bin_energy=np.array([1.0, 0.7]))
    with pytest.raises(RuntimeError):
        orc.trace(tree, [src], o, 10, seed=1, poly_group=2)
