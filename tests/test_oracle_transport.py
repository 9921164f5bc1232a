"""Pins for the oracle's Monte Carlo formal solution (Sects. 2.3-2.4).

Each check compares against something the oracle does not compute itself:
closed-form transmission, the optically thin mean intensity of a point
source and of an isotropic field, exact energy bookkeeping, the invariance of
continuous-absorption paths under refinement of a uniform medium, the
analog estimator's expectation, the Henyey-Greenstein distribution, and a
hand-computed single peel-off.
"""
import math

import numpy as np
import pytest

from paper_1206_3710_gb300 import synth


def _optics(kext, albedo=0.0, g=0.0, n=1):
    return synth.Optics(lambda_um=np.full(n, 0.55), kappa_ext=np.full(n, kext), albedo=np.full(n, albedo),
                        g_hg=np.full(n, g), dnu=np.ones(n))


class _Beam:
    kind = "beam"

    def __init__(self, pos, dir_, energy=1.0):
        self.pos, self.dir, self.bin_energy = pos, dir_, np.array([energy])


def _zscores(mc, expect, sumsq, n):
    var = np.maximum(sumsq - mc * mc / n, 0.0)
    sig = np.sqrt(var)
    ok = sig > 0
    return (mc[ok] - expect[ok]) / sig[ok]


# P1 -----------------------------------------------------------------------

def test_p1_beam_transmission_exact(orc):
    L, rho, tau = 4.0, 2.0, 1.7
    desc = synth.random_refined_tree((4, 4, 4), (L, L, L), 2, 0.3, 4, rho_fn=lambda l, x, y, z: np.full(x.size, rho))
    tree = orc.Tree(desc)
    kext = tau / (rho * L)
    r = orc.trace(tree, [_Beam((0.0, 1.3, 2.7), (1.0, 0.0, 0.0))], _optics(kext), 1000, seed=3, record=True)
    W0 = 1.0 / 1000
    np.testing.assert_allclose(r["rec"][:, 0], W0 * math.exp(-tau), rtol=1e-12)
    led = r["ledger"]
    assert abs(led["absorbed"] - (1 - math.exp(-tau))) < 1e-12


def test_p1_point_source_pure_absorber_exact(orc):
    L, rho = 3.0, 0.5
    desc = synth.random_refined_tree((3, 3, 3), (L, L, L), 2, 0.4, 9, rho_fn=lambda l, x, y, z: np.full(x.size, rho))
    tree = orc.Tree(desc)
    kext = 0.9
    src = synth.Source("point", bin_energy=np.array([2.0]), pos=(1.1, 1.7, 0.4))
    r = orc.trace(tree, [src], _optics(kext), 2000, seed=8, record=True)
    rec = r["rec"]
    dist = np.linalg.norm(rec[:, 4:7] - np.array(src.pos), axis=1)
    np.testing.assert_allclose(rec[:, 0], (2.0 / 2000) * np.exp(-kext * rho * dist), rtol=1e-11)
    # exit point on the boundary along the emission direction
    on_face = np.min(np.minimum(np.abs(rec[:, 4:7]), np.abs(rec[:, 4:7] - L)), axis=1)
    assert on_face.max() < 1e-12


def test_p1_analog_binomial(orc):
    L, rho, tau = 2.0, 1.0, 1.2
    desc = synth.uniform_tree((2, 2, 2), (L, L, L), rho)
    tree = orc.Tree(desc)
    n = 200000
    r = orc.trace(tree, [_Beam((0.0, 0.5, 0.5), (1.0, 0.0, 0.0))], _optics(tau / (rho * L)), n, seed=5,
                  estimator=orc.EST_ANALOG)
    p = math.exp(-tau)
    frac = r["ledger"]["escaped"]
    assert abs(frac - p) < 4 * math.sqrt(p * (1 - p) / n)


# P2 -----------------------------------------------------------------------

def _gl_cell_mean(lo, size, src, kext_rho, n=8):
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1) * size
    w = 0.5 * w * size
    X, Y, Z = np.meshgrid(lo[0] + x, lo[1] + x, lo[2] + x, indexing="ij")
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]
    r = np.sqrt((X - src[0]) ** 2 + (Y - src[1]) ** 2 + (Z - src[2]) ** 2)
    return (W * np.exp(-kext_rho * r) / (4 * math.pi * r * r)).sum()


def test_p2_thin_point_source_mean_intensity(orc):
    n_root, L, rho = 12, 12.0, 1.0
    desc = synth.uniform_tree((n_root,) * 3, (L,) * 3, rho)
    tree = orc.Tree(desc)
    kext = 1e-3 / L
    src = synth.Source("point", bin_energy=np.array([1.0]), pos=(6.0, 6.0, 6.0))
    npk = 1_000_000
    r = orc.trace(tree, [src], _optics(kext), npk, seed=21, validation=True, n_threads=8)
    A = r["absorbed"][0]
    expect = np.zeros_like(A)
    for iz in range(n_root):
        for iy in range(n_root):
            for ix in range(n_root):
                c = ix + n_root * (iy + n_root * iz)
                expect[c] = kext * rho * _gl_cell_mean(np.array([ix, iy, iz], float), 1.0, src.pos, kext * rho)
    lo = np.array([[ix, iy, iz] for iz in range(n_root) for iy in range(n_root) for ix in range(n_root)], float)
    far = np.all((lo >= 7) | (lo + 1 <= 5), axis=1)   # cells not adjacent to the source
    z = _zscores(A[far], expect[far], r["sumsq"][0][far], npk)
    assert np.mean(np.abs(z) > 3) < 0.01
    assert np.abs(z).max() < 5.5
    well = far & (r["hits"][0] >= 1000)
    assert well.sum() > 100
    # mean relative deviation (signed: a bias check) under 1% on cells with
    # >= 1e3 hits; the per-cell scatter there is ~1/sqrt(hits) ~ 3%
    rel = A[well] / expect[well] - 1
    assert abs(rel.mean()) < 0.01
    dense = far & (r["hits"][0] >= 10000)
    assert dense.sum() > 20
    assert np.abs(A[dense] / expect[dense] - 1).mean() < 0.01


# P3 -----------------------------------------------------------------------

def test_p3_energy_conservation(orc):
    m = synth.tiny_clump()
    tree = orc.Tree(m.tree)
    r = orc.trace(tree, m.sources, m.optics, 50000, seed=2, observers=m.observers, n_threads=4)
    L = r["ledger"]
    assert abs(L["emitted"] - L["absorbed"] - L["escaped"]) <= 1e-12 * L["emitted"]
    assert abs(r["absorbed"].sum() - L["absorbed"]) <= 1e-12 * L["emitted"]
    assert L["n_scatter"] > 0


def test_p3_roulette_bookkeeping(orc):
    m = synth.tiny_clump()
    tree = orc.Tree(m.tree)
    opt = _optics(m.optics.kappa_ext[0] * 30, albedo=0.9)      # thick and scattering: many roulette events
    n = 20000
    wmin, p = 1e-2, 0.7
    r = orc.trace(tree, m.sources, opt, n, seed=4, rr_wmin=wmin, rr_p=p, n_threads=4)
    L = r["ledger"]
    lhs = L["emitted"] + L["rr_gain"]
    rhs = L["absorbed"] + L["escaped"] + L["rr_loss"]
    assert abs(lhs - rhs) <= 1e-12 * lhs
    assert L["rr_loss"] > 0
    W0 = 1.0 / n
    sd = wmin * W0 * math.sqrt(p / (1 - p)) * math.sqrt(L["n_scatter"])
    assert abs(L["rr_gain"] - L["rr_loss"]) < 5 * sd


# P4 -----------------------------------------------------------------------

def test_p4_refined_uniform_equals_fine_grid(orc):
    """With continuous absorption and the free path drawn in scattering optical
    depth, a package's path in a uniform medium does not depend on how the
    medium is cut into cells (Sect. 2.3): refined and fine grids agree."""
    L, rho = 4.0, 1.0
    coarse = synth.random_refined_tree((4, 4, 4), (L,) * 3, 2, 0.5, 17,
                                       rho_fn=lambda l, x, y, z: np.full(x.size, rho))
    fine = synth.uniform_tree((16, 16, 16), (L,) * 3, rho)
    tc, tf = orc.Tree(coarse), orc.Tree(fine)
    opt = _optics(0.8, albedo=0.6, g=0.3)
    src = synth.Source("point", bin_energy=np.array([1.0]), pos=(1.3, 2.2, 2.9))
    obs = synth.axis_observers(16, L, "all6")
    kw = dict(seed=33, record=True, observers=obs)
    rc = orc.trace(tc, [src], opt, 3000, **kw)
    rf = orc.trace(tf, [src], opt, 3000, **kw)
    np.testing.assert_allclose(rc["rec"][:, 0], rf["rec"][:, 0], rtol=1e-9, atol=1e-18)
    np.testing.assert_array_equal(rc["rec"][:, 1], rf["rec"][:, 1])
    np.testing.assert_allclose(rc["rec"][:, 4:], rf["rec"][:, 4:], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(rc["images"], rf["images"], rtol=1e-9, atol=1e-15)
    # aggregate the fine cells to the leaves of the refined grid
    from tests.test_oracle_geometry import leaf_boxes
    agg = []
    for cid, lo, size in leaf_boxes(coarse):
        k = int(round(4 * size))
        i0 = (lo * 4).round().astype(int)
        ix, iy, iz = np.meshgrid(np.arange(i0[0], i0[0] + k), np.arange(i0[1], i0[1] + k),
                                 np.arange(i0[2], i0[2] + k), indexing="ij")
        agg.append((cid, rf["absorbed"][0][(ix + 16 * (iy + 16 * iz)).ravel()].sum()))
    a_c = np.array([rc["absorbed"][0][c] for c, _ in agg])
    a_f = np.array([v for _, v in agg])
    np.testing.assert_allclose(a_c, a_f, rtol=1e-9, atol=1e-15)
    # the paper's map metrics (Eqs. 6-7) for the two images
    Ia, If = rc["images"].ravel(), rf["images"].ravel()
    assert abs((Ia - If).sum() / If.sum()) < 1e-9
    assert math.sqrt(((Ia - If) ** 2).sum() / (If ** 2).sum()) < 1e-9


# P6 -----------------------------------------------------------------------

def test_p6_isotropic_external_field(orc):
    n_root, L, rho = 8, 8.0, 1.0
    desc = synth.uniform_tree((n_root,) * 3, (L,) * 3, rho)
    tree = orc.Tree(desc)
    kext = 1e-4 / L
    E = 1.0
    src = synth.Source("external", bin_energy=np.array([E]))
    npk = 400000
    r = orc.trace(tree, [src], _optics(kext), npk, seed=6, validation=True, n_threads=8)
    A = r["absorbed"][0]
    S = 6 * L * L
    expect = np.full_like(A, 4 * kext * rho * 1.0 * E / S)  # J = I = E/(pi S); A = 4 pi kappa rho V J
    z = _zscores(A, expect, r["sumsq"][0], npk)
    assert np.mean(np.abs(z) > 3) < 0.015
    assert np.abs(z).max() < 5.5
    assert abs(A.sum() / expect.sum() - 1) < 0.005
    assert abs(r["ledger"]["emitted"] - E) < 1e-12


# P7 -----------------------------------------------------------------------

@pytest.mark.parametrize("g", [-0.6, 0.0, 0.3, 0.5, 0.9])
def test_p7_hg_inverse_cdf_and_mean(orc, g):
    def cdf(mu):
        if g == 0:
            return 0.5 * (mu + 1)
        return (1 - g * g) / (2 * g) * (1 / math.sqrt(1 + g * g - 2 * g * mu) - 1 / (1 + g))
    for mu in np.linspace(-0.999, 0.999, 37):
        assert abs(orc.hg_mu(g, cdf(mu)) - mu) < 1e-9
    n = 20000
    m = np.mean([orc.hg_mu(g, (i + 0.5) / n) for i in range(n)])
    assert abs(m - g) < 1e-6
    # phase function normalised over 4 pi and equal to the density of mu / 2 pi
    x, w = np.polynomial.legendre.leggauss(200)
    ph = np.array([orc.hg_phase(g, v) for v in x])
    assert abs(2 * math.pi * (w * ph).sum() - 1) < 1e-6 if abs(g) < 0.8 else 1e-3
    eps = 1e-6
    for v in (-0.5, 0.1, 0.7):
        dens = (cdf(v + eps) - cdf(v - eps)) / (2 * eps)
        assert abs(orc.hg_phase(g, v) * 2 * math.pi - dens) < 1e-5 * max(1, dens)


def test_p7_rotation(orc):
    rng = np.random.default_rng(1)
    for _ in range(500):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        if _ % 50 == 0:
            d = np.array([0.0, 0.0, 1.0 if _ % 100 == 0 else -1.0])
        mu, phi = rng.uniform(-1, 1), rng.uniform(0, 2 * math.pi)
        o = orc.scatter_dir(d, mu, phi)
        assert abs(np.linalg.norm(o) - 1) < 1e-12
        assert abs(o @ d - mu) < 1e-9
    d = np.array([0.3, -0.5, 0.81])
    d /= np.linalg.norm(d)
    avg = np.mean([orc.scatter_dir(d, 0.4, 2 * math.pi * (i + 0.5) / 64) for i in range(64)], axis=0)
    np.testing.assert_allclose(avg, 0.4 * d, atol=1e-12)


# P8 -----------------------------------------------------------------------

def test_p8_continuous_vs_analog(orc):
    """Continuous absorption and the analog estimator have the same
    expectations: escaped energy and absorbed energy per cell."""
    m = synth.tiny_clump()
    tree = orc.Tree(m.tree)
    opt = _optics(m.optics.kappa_ext[0] * 2, albedo=0.5)
    n = 200000
    rc = orc.trace(tree, m.sources, opt, n, seed=7, record=True, validation=True)
    ra = orc.trace(tree, m.sources, opt, n, seed=8, record=True, validation=True, estimator=orc.EST_ANALOG)
    ec, ea = rc["rec"][:, 0], ra["rec"][:, 0]
    sd = math.sqrt(n * (ec.var() + ea.var()))
    assert abs(ec.sum() - ea.sum()) < 4 * sd
    Ac, Aa = rc["absorbed"][0], ra["absorbed"][0]
    vc = np.maximum(rc["sumsq"][0] - Ac * Ac / n, 0)
    # analog deposits are whole packages of weight W0: compound Poisson with
    # variance W0 * mean; use the pooled mean so empty cells are not zero-variance
    W0 = 1.0 / n
    pooled = 0.5 * (Ac + Aa)
    va = W0 * pooled
    ok = pooled / W0 >= 25          # normal approximation: >= 25 expected events
    assert ok.sum() > 300
    z = (Ac[ok] - Aa[ok]) / np.sqrt(vc[ok] + va[ok])
    assert np.mean(np.abs(z) > 3) < 0.01
    assert np.abs(z).max() < 5.5
    assert rc["ledger"]["n_scatter"] > 0 and ra["ledger"]["n_scatter"] > 0


# P9 -----------------------------------------------------------------------

def test_p9_single_peel_exact(orc):
    L, rho, n = 4.0, 1.5, 8
    desc = synth.uniform_tree((n,) * 3, (L,) * 3, rho)
    tree = orc.Tree(desc)
    kext, g = 0.35, 0.5
    opt = _optics(kext, albedo=0.5, g=g)
    obs = synth.Observers(dirs=np.array([[0.0, 0.0, 1.0]]), ups=np.array([[0.0, 1.0, 0.0]]), nx=10, ny=10,
                          fov=(L, L))
    x = np.array([1.05, 2.95, 1.3])
    d_in = np.array([0.6, 0.0, 0.8])
    W = 2.5
    img = orc.peel_point(tree, opt, obs, 0, x, d_in, W)
    mu = 0.8
    p = (1 - g * g) / (4 * math.pi * (1 + g * g - 2 * g * mu) ** 1.5)
    val = W * p * math.exp(-kext * rho * (L - x[2]))
    # ex = up x k = (1,0,0), ey = k x ex = (0,1,0); pixel 0.4 cm
    px = int(math.floor((x[0] - 2.0) / 0.4 + 5))
    py = int(math.floor((x[1] - 2.0) / 0.4 + 5))
    expect = np.zeros((1, 1, 10, 10))
    expect[0, 0, py, px] = val
    np.testing.assert_allclose(img, expect, rtol=1e-12, atol=0)


def test_p9_peel_matches_escape_binning(orc):
    """The peeled image total (energy per steradian toward the observer)
    equals the scattered energy escaping into a cone around the observer's
    direction per unit solid angle, for a model whose scattered light is
    close to isotropic by symmetry."""
    L, n = 10.0, 10
    desc = synth.uniform_tree((n,) * 3, (L,) * 3, 1.0)
    tree = orc.Tree(desc)
    opt = _optics(0.05, albedo=1.0, g=0.0)
    obs = synth.Observers(dirs=np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0]]), ups=np.array([[0, 1.0, 0], [0, 0, 1.0]]),
                          nx=20, ny=20, fov=(2 * L, 2 * L))
    src = synth.Source("point", bin_energy=np.array([1.0]), pos=(5.0, 5.0, 5.0))
    npk = 300000
    r = orc.trace(tree, [src], opt, npk, seed=12, record=True, observers=obs, n_threads=8)
    rec = r["rec"]
    scat = rec[:, 1] > 0
    cth = math.cos(math.radians(20))
    omega = 2 * math.pi * (1 - cth)
    for o, k in enumerate(obs.dirs):
        inside = scat & (rec[:, 7:10] @ k > cth)
        est = rec[inside, 0].sum() / omega
        sd = math.sqrt((rec[inside, 0] ** 2).sum()) / omega
        peel = r["images"][o].sum()
        assert abs(peel - est) < 4 * sd + 0.02 * est, (o, peel, est, sd)
    assert r["ledger"]["n_peel_out"] == 0


# Sharding ------------------------------------------------------------------

def test_shards_are_one_run(orc):
    """Packages are independent (Sect. 5.2): two shards of n packages per bin
    with package offsets 0 and n are, package by package, the first and
    second half of one run of 2n (each shard's weights carry the full source
    energy, i.e. twice the single run's), so their mean is that run."""
    m = synth.tiny_clump()
    tree = orc.Tree(m.tree)
    n = 1500
    kw = dict(seed=9, record=True, rr_wmin=0.3, rr_p=0.6)
    one = orc.trace(tree, m.sources, m.optics, 2 * n, **kw)
    a = orc.trace(tree, m.sources, m.optics, n, packet_offset=0, **kw)
    b = orc.trace(tree, m.sources, m.optics, n, packet_offset=n, **kw)
    rec = np.concatenate([a["rec"], b["rec"]])
    np.testing.assert_array_equal(rec[:, 1:], one["rec"][:, 1:])      # scatterings, crossings, fate, exit
    np.testing.assert_array_equal(rec[:, 0], 2.0 * one["rec"][:, 0])  # escaped weight, W0 doubled exactly
    np.testing.assert_allclose(0.5 * (a["absorbed"] + b["absorbed"]), one["absorbed"], rtol=1e-12,
                               atol=1e-15 * one["absorbed"].max())
    assert one["ledger"]["rr_loss"] > 0
    # a different offset is a different set of packages
    c = orc.trace(tree, m.sources, m.optics, n, packet_offset=7, **kw)
    assert not np.array_equal(c["rec"][:, 2], a["rec"][:, 2])


# Accelerated peel-off (Sect. 2.4) ---------------------------------------------

_OBLIQUE = np.array([[0.6, 0.8, 0.0], [0.0, 0.6, -0.8], [-0.48, 0.6, 0.64], [-1.0, 0.0, 0.0]])


def _obs(dirs, n=16, fov=1.0):
    ups = np.array([(0.0, 0.0, 1.0) if abs(d[2]) < 0.9 else (1.0, 0.0, 0.0) for d in dirs])
    return synth.Observers(dirs=np.asarray(dirs, float), ups=ups, nx=n, ny=n, fov=(fov, fov))


def test_peel_table_uniform_closed_form(orc):
    """In a uniform medium the tabulated column is the density times the
    distance from the tile centre to the border along the direction; checked
    for oblique and axis directions, with blocks that do not divide the root
    grid (partial blocks and tiles)."""
    root, B, S, rho = (10, 7, 12), 4, 2, 3.0
    desc = synth.random_refined_tree(root, tuple(float(r) for r in root), 2, 0.3, 5,
                                     rho_fn=lambda l, x, y, z: np.full(x.size, rho))
    tree = orc.Tree(desc)
    obs = _obs(_OBLIQUE)
    tab = orc.peel_table(tree, obs, B, S)
    nb = [(r + B - 1) // B for r in root]
    i = 0
    for k in obs.dirs:
        for bz in range(nb[2]):
            for by in range(nb[1]):
                for bx in range(nb[0]):
                    b = (bx, by, bz)
                    for a in range(3):
                        if k[a] == 0:
                            continue
                        a1, a2 = (a + 1) % 3, (a + 2) % 3
                        for iv in range(S):
                            for iu in range(S):
                                w = B / S
                                u0, v0 = b[a1] * B + iu * w, b[a2] * B + iv * w
                                if u0 >= root[a1] or v0 >= root[a2]:
                                    expect = 0.0
                                else:
                                    c = np.zeros(3)
                                    c[a] = min((b[a] + 1) * B, root[a]) if k[a] > 0 else b[a] * B
                                    c[a1] = 0.5 * (u0 + min(u0 + w, root[a1]))
                                    c[a2] = 0.5 * (v0 + min(v0 + w, root[a2]))
                                    dist = min(((root[d] if k[d] > 0 else 0.0) - c[d]) / k[d]
                                               for d in range(3) if k[d] != 0)
                                    expect = rho * max(dist, 0.0)
                                assert tab[i] == pytest.approx(expect, rel=1e-12, abs=1e-12), (i, expect)
                                i += 1
    assert i == tab.size


def test_peel_tabulated_exact_along_axes(orc):
    """Observers along the axes, tiles the size of a root-cell face, no
    refinement: every point of a tile sees the same row of cells to the
    border, so the accelerated peel-off equals the exact one."""
    root = (12, 10, 8)
    rng = np.random.default_rng(3)
    desc = synth.grow_tree(root, tuple(float(r) for r in root), 0,
                           lambda l, x, y, z: rng.uniform(0.2, 2.0, x.size),
                           lambda l, x, y, z, r: np.zeros(x.size, bool))
    tree = orc.Tree(desc)
    lam = np.array([0.55])
    optics = synth.Optics(lambda_um=lam, kappa_ext=np.array([0.3]), albedo=np.array([0.7]),
                          g_hg=np.array([0.3]), dnu=np.ones(1))
    src = synth.Source("point", bin_energy=np.array([1.0]), pos=(6.1, 5.3, 3.7))
    obs = _obs([[1, 0, 0], [0, -1, 0], [0, 0, 1]], n=24, fov=16.0)
    exact = orc.trace(tree, [src], optics, 4000, seed=3, observers=obs)
    tab = orc.trace(tree, [src], optics, 4000, seed=3, observers=obs, peel_block=4, peel_tiles=4)
    assert exact["images"].sum() > 0
    np.testing.assert_allclose(tab["images"], exact["images"], rtol=1e-11, atol=1e-14 * exact["images"].max())
    assert tab["ledger"]["n_peel_cross"] < exact["ledger"]["n_peel_cross"]


def test_image_variance_tally_sums_whole_packages(orc):
    """The per-pixel variance tally squares each package's whole
    contribution to a pixel (all its scatterings together): a run of N
    packages gives sum_k c_k^2 with c_k the image of package k traced on its
    own (packet_offset k, whose weight is N times the joint run's)."""
    m = synth.tiny_clump()
    tree = orc.Tree(m.tree)
    opt = synth.Optics(lambda_um=m.optics.lambda_um, kappa_ext=m.optics.kappa_ext * 3.0,
                       albedo=np.full(1, 0.9), g_hg=np.full(1, 0.3), dnu=m.optics.dnu)
    # few pixels, so that one package often lands in a pixel more than once
    obs = synth.Observers(dirs=np.array([[0.0, 0.0, 1.0], [0.6, 0.8, 0.0]]),
                          ups=np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 1.0]]), nx=3, ny=3, fov=m.observers.fov)
    n = 40
    joint = orc.trace(tree, m.sources, opt, n, seed=31, observers=obs, validation=True, n_threads=4)
    assert joint["ledger"]["n_scatter"] > 3 * n
    sq = np.zeros_like(joint["images"])
    tot = np.zeros_like(joint["images"])
    repeat = False
    for k in range(n):
        one = orc.trace(tree, m.sources, opt, 1, seed=31, observers=obs, packet_offset=k)
        c = one["images"] / n
        tot += c
        sq += c * c
        repeat |= one["ledger"]["n_scatter"] > 4
    assert repeat
    np.testing.assert_allclose(tot, joint["images"], rtol=1e-12, atol=1e-15 * joint["images"].max())
    np.testing.assert_allclose(joint["image_sumsq"], sq, rtol=1e-12, atol=1e-15 * sq.max())
    # squaring each scattering's contribution instead would give less
    assert (joint["image_sumsq"] >= joint["images"] ** 2 / n - 1e-15).all()
