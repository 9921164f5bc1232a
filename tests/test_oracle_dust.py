"""Pins for the oracle's dust-temperature solve and Lambda iteration
(Sect. 3.1 Eq. 2, Sect. 3.2, and the single-component equilibrium dust of
Sect. 4)."""
import math

import pytest

import numpy as np

from paper_1206_3710_gb300 import synth

SIGMA_SB = 5.670374419e-5


def test_p10_round_trip(orc):
    desc = synth.random_refined_tree((3, 3, 3), (3e16,) * 3, 2, 0.3, 5,
                                     rho_fn=lambda l, x, y, z: np.random.default_rng(l).uniform(1e-22, 1e-20, x.size))
    tree = orc.Tree(desc)
    lev, leaf = tree.cells()
    lam = synth.log_lambda_grid(30)
    kabs = 200.0 * (lam / 0.55) ** -1.8
    dnu = synth.bin_dnu(lam)
    rng = np.random.default_rng(3)
    T_true = rng.uniform(5.0, 2000.0, tree.n_cells)
    V = (desc.box[0] / desc.root[0] * 0.5 ** lev.astype(float)) ** 3
    A = np.array([desc.density[i] * V[i] * orc.emission_per_mass(lam, kabs, dnu, T_true[i])
                  for i in range(tree.n_cells)])
    T = orc.dust_temperature(tree, A, lam, kabs, dnu, n_threads=4)
    np.testing.assert_allclose(T[leaf], T_true[leaf], rtol=1e-10)
    assert np.all(T[~leaf] == 0)
    # clamping at the bounds
    T2 = orc.dust_temperature(tree, np.zeros(tree.n_cells), lam, kabs, dnu)
    assert np.all(T2[leaf] == 2.7)


def test_p10_grey_planck_integral(orc):
    """Grey opacity with a dense wavelength grid: the quadrature reproduces
    the full Planck integral, sum B_nu dnu = sigma T^4 / pi, so the
    equilibrium temperature is (A / (4 sigma kappa rho V))^(1/4)."""
    lam = np.logspace(-2, 5, 4000)
    kappa = 50.0
    kabs = np.full(lam.size, kappa)
    dnu = synth.bin_dnu(lam)
    for T in (10.0, 30.0, 100.0, 300.0, 1000.0):
        E = orc.emission_per_mass(lam, kabs, dnu, T)
        assert abs(E / (4 * kappa * SIGMA_SB * T ** 4) - 1) < 1e-4, T
    desc = synth.uniform_tree((2, 2, 2), (2e16,) * 3, 1e-20)
    tree = orc.Tree(desc)
    V = 1e48
    T_exp = np.array([15.0, 40.0, 80.0, 120.0, 300.0, 500.0, 800.0, 1000.0])
    A = 4 * SIGMA_SB * kappa * 1e-20 * V * T_exp ** 4
    T = orc.dust_temperature(tree, A, lam, kabs, dnu)
    np.testing.assert_allclose(T, T_exp, rtol=1e-4)


def test_p10_emission_monotone_and_scaling(orc):
    lam = synth.log_lambda_grid(20)
    kabs = (lam / 0.55) ** -1.8
    dnu = synth.bin_dnu(lam)
    Ts = np.logspace(0.5, 3.4, 50)
    E = np.array([orc.emission_per_mass(lam, kabs, dnu, t) for t in Ts])
    assert np.all(np.diff(E) > 0)
    # linear in kappa
    assert abs(orc.emission_per_mass(lam, 3 * kabs, dnu, 50.0) / orc.emission_per_mass(lam, kabs, dnu, 50.0) - 3) < 1e-14


def _small_star_model(tau_scale):
    L = 20 * synth.AU_CM
    n = 8
    rho = 1e-18
    desc = synth.uniform_tree((n,) * 3, (L,) * 3, rho)
    lam = synth.log_lambda_grid(12)
    kappa1 = tau_scale / (rho * L)
    optics = synth.powerlaw_dust(lam, kappa1, 1.0)
    Lb = synth.blackbody_star_bins(lam, 4000.0, 2 * synth.RSUN_CM)
    star = synth.Source("point", bin_energy=Lb, pos=(0.5 * L,) * 3)
    return desc, optics, star


def test_p12_lambda_iteration_thin_limit(orc):
    """Optically thin to its own emission: the Lambda iteration stops at once
    and the temperature equals the single-pass (star only) temperature."""
    desc, optics, star = _small_star_model(1e-4)
    tree = orc.Tree(desc)
    T, hist = orc.lambda_iterate(tree, star, optics, 20000, 20000, seed=9, tol=1e-3, min_hits=100, n_threads=4)
    kabs = (1 - optics.albedo) * optics.kappa_ext
    r = orc.trace(tree, [star], optics, 20000, seed=9, per_lambda=False)
    T1 = orc.dust_temperature(tree, r["absorbed"][0], optics.lambda_um, kabs, optics.dnu)
    assert len(hist) == 1
    np.testing.assert_allclose(T, T1, rtol=1e-3)


def test_p12_lambda_iteration_self_heating(orc):
    """With dust optically thick to its own emission, the iteration raises
    the temperatures (dust heats dust) and dT/T shrinks with each step.  At
    convergence the fixed point of Eq. 2 holds, checked with random numbers
    the iteration never used:
      * per cell, the dust's emission at the final T equals the energy it
        absorbs from the star plus from a fresh trace of that emission
        (independent streams), within the Monte Carlo error;
      * in total, everything the star emits leaves the box: the energy the
        dust absorbed from the star equals what its own emission loses
        through the boundary (emitted minus re-absorbed)."""
    desc, optics, star = _small_star_model(3.0)
    tree = orc.Tree(desc)
    level, leaf = tree.cells()
    kabs = (1 - optics.albedo) * optics.kappa_ext
    lam, dnu = optics.lambda_um, optics.dnu
    n = 40000
    r = orc.trace(tree, [star], optics, n, seed=4, per_lambda=False, validation=True, n_threads=8)
    T0 = orc.dust_temperature(tree, r["absorbed"][0], lam, kabs, dnu)
    T, hist = orc.lambda_iterate(tree, star, optics, n, n, seed=4, tol=1e-4, max_iter=40, min_hits=50,
                                 n_threads=8)
    assert np.median(T[leaf] / T0[leaf]) > 1.01
    assert hist[-1] < hist[0] and hist[-1] < 1e-4 and len(hist) >= 2
    # a fresh dust trace at the final temperatures (another seed)
    em = orc.dust_emission(tree, T, lam, kabs, dnu)
    npk = orc.packets_by_energy(em.sum(axis=1), n)
    rd = orc.trace(tree, [orc._DustSource(em)], optics, npk, seed=1234, iter_=1, per_lambda=False,
                   validation=True, n_threads=8)
    A = r["absorbed"][0] + rd["absorbed"][0]
    E = em.sum(axis=0)                       # emission per cell (energy per unit time)
    n_d = int(npk.sum())
    var = (np.maximum(r["sumsq"][0] - r["absorbed"][0] ** 2 / (n * lam.size), 0)
           + np.maximum(rd["sumsq"][0] - rd["absorbed"][0] ** 2 / n_d, 0))
    hits = r["hits"][0] + rd["hits"][0]
    ok = leaf & (hits >= 1000) & (var > 0)
    assert ok.sum() > 0.8 * leaf.sum()
    z = (E[ok] - A[ok]) / np.sqrt(var[ok])
    assert np.mean(np.abs(z) > 3) < 0.02, np.sort(np.abs(z))[-5:]
    assert abs(np.mean(E[ok] / A[ok] - 1)) < 0.01
    # global: absorbed from the star = dust emission that escapes
    Ld = rd["ledger"]
    absorbed_star = r["ledger"]["absorbed"]
    escaped_dust = Ld["emitted"] - Ld["absorbed"]
    assert abs(escaped_dust / absorbed_star - 1) < 0.01, (escaped_dust, absorbed_star)
    # the pin has teeth: the star's field alone is far from this balance
    E0 = orc.dust_emission(tree, T0, lam, kabs, dnu).sum(axis=0)
    assert np.mean(np.abs(E0[ok] / A[ok] - 1)) > 0.05


# P13: subiterations (Sect. 3.2, App. B) --------------------------------------

def _sub_model(tau=2.0):
    L = 20 * synth.AU_CM
    desc = synth.random_refined_tree((6, 6, 6), (L,) * 3, 3, 0.35, 21,
                                     rho_fn=lambda l, x, y, z: np.random.default_rng(l + 3).uniform(0.5e-18, 2e-18,
                                                                                                    x.size))
    lam = synth.log_lambda_grid(8)
    optics = synth.powerlaw_dust(lam, tau / (1e-18 * L), 1.0)
    star = synth.Source("point", bin_energy=synth.blackbody_star_bins(lam, 4000.0, 2 * synth.RSUN_CM),
                        pos=(0.43 * L, 0.52 * L, 0.47 * L))
    return desc, optics, star


def _dust_source(orc, tree, optics, T):
    kabs = (1 - optics.albedo) * optics.kappa_ext
    return orc.dust_emission(tree, T, optics.lambda_um, kabs, optics.dnu)


def test_p13_levels_partition_the_field(orc):
    """Splitting the dust field by the shallowest grid level a package reached
    changes where deposits are summed, not what is deposited: the level
    arrays add up to the plain field, and a cell holds nothing above its own
    level (a package in a cell has been in that cell's grid)."""
    desc, optics, _ = _sub_model()
    tree = orc.Tree(desc)
    level, leaf = tree.cells()
    T = np.where(leaf, 300.0 * np.random.default_rng(2).uniform(0.5, 1.5, tree.n_cells), 0.0)
    em = _dust_source(orc, tree, optics, T)
    src = orc._DustSource(em)
    plain = orc.trace(tree, [src], optics, 3000, seed=8, iter_=1, per_lambda=False)
    lev = orc.trace(tree, [src], optics, 3000, seed=8, iter_=1, per_lambda=False, per_level=True)
    A = lev["absorbed"]
    assert A.shape == (desc.n_levels, tree.n_cells)
    np.testing.assert_allclose(A.sum(axis=0), plain["absorbed"][0], rtol=1e-12, atol=1e-14 * plain["absorbed"].max())
    for i in range(desc.n_levels):
        assert np.all(A[i][level < i] == 0)
    assert all(A[i].sum() > 0 for i in range(desc.n_levels))
    assert lev["ledger"]["n_cross"] == plain["ledger"]["n_cross"]


def test_p13_confinement(orc):
    """Confined to the subtrees below level L, packages emitted there deposit
    only into levels > L, and whatever leaves a subtree is booked as escaped
    (the energy balance still closes)."""
    desc, optics, _ = _sub_model()
    tree = orc.Tree(desc)
    level, leaf = tree.cells()
    L = 0
    T = np.where(leaf & (level > L), 250.0, 0.0)
    em = _dust_source(orc, tree, optics, T)
    r = orc.trace(tree, [orc._DustSource(em)], optics, 3000, seed=8, iter_=1, per_lambda=False, per_level=True,
                  confine_level=L)
    A = r["absorbed"]
    assert np.all(A[:L + 1] == 0) and A[L + 1:].sum() > 0
    assert np.all(A.sum(axis=0)[level <= L] == 0)
    led = r["ledger"]
    assert abs(led["emitted"] - led["absorbed"] - led["escaped"]) <= 1e-12 * led["emitted"]
    free = orc.trace(tree, [orc._DustSource(em)], optics, 3000, seed=8, iter_=1, per_lambda=False)
    assert led["escaped"] > free["ledger"]["escaped"]


def test_p13_full_schedule_is_the_lambda_iteration(orc):
    """With full steps only, the subiteration driver is the Lambda iteration
    of Eq. 2: the same temperatures and changes step by step."""
    desc, optics, star = _sub_model()
    tree = orc.Tree(desc)
    T1, h1 = orc.lambda_iterate(tree, star, optics, 2000, 2000, seed=6, tol=0.0, max_iter=3, min_hits=10)
    T2, h2, _ = orc.lambda_subiterate(tree, star, optics, 2000, 2000, seed=6, schedule=["full"] * 3, sub_level=1,
                                      min_hits=10)
    np.testing.assert_allclose(T2, T1, rtol=1e-12)
    np.testing.assert_allclose(h2, h1, rtol=1e-9)


def test_p13_self_absorption_and_ali(orc):
    """The diagonal of Lambda (Eq. 3): in a one-cell model every dust deposit
    lands in the package's own emission cell, so the self-absorption tally
    equals the absorbed dust energy; and the ALI step, which solves for the
    cell's own re-absorption, converges where the plain Lambda iteration
    (Eq. 2) still creeps upwards."""
    L = 5 * synth.AU_CM
    rho = 1e-18
    desc = synth.uniform_tree((1, 1, 1), (L,) * 3, rho)
    tree = orc.Tree(desc)
    lam = synth.log_lambda_grid(10)
    o = synth.powerlaw_dust(lam, 2000.0 / (rho * L), 1.0)   # thick to its own emission, a pure absorber
    optics = synth.Optics(o.lambda_um, o.kappa_ext, np.zeros(lam.size), np.zeros(lam.size), o.dnu)
    star = synth.Source("point", bin_energy=synth.blackbody_star_bins(lam, 4000.0, 2 * synth.RSUN_CM),
                        pos=(0.5 * L, 0.51 * L, 0.49 * L))
    kabs = (1 - optics.albedo) * optics.kappa_ext
    T0 = np.array([100.0])
    em = orc.dust_emission(tree, T0, optics.lambda_um, kabs, optics.dnu)
    self_abs = np.zeros((lam.size, 1))
    r = orc.trace(tree, [orc._DustSource(em)], optics, 4000, seed=2, iter_=1, per_lambda=True,
                  self_absorbed=self_abs)
    np.testing.assert_allclose(self_abs[:, 0], r["absorbed"][:, 0], rtol=1e-12)
    assert self_abs.sum() > 0
    kw = dict(seed=3, schedule=["full"] * 5, sub_level=0, min_hits=0.0, dust_per_bin=True)
    T_plain, h_plain, _ = orc.lambda_subiterate(tree, star, optics, 2000, 2000, **kw)
    T_ali, h_ali, _ = orc.lambda_subiterate(tree, star, optics, 2000, 2000, ali=True, **kw)
    assert h_plain[3] > 0.02 and h_ali[3] < 0.25 * h_plain[3]
    assert T_ali[0] > T_plain[0]   # the plain iteration is still climbing towards it


def test_p13_self_absorption_bounded(orc):
    """The two tallies behind Lambda_cc: what a cell's own packages leave in
    it is part of what it absorbed and of what they carried; the carried
    energies add up to the whole dust emission (every package is booked at
    its emission cell once), and per cell they follow the emission."""
    desc, optics, _ = _sub_model()
    tree = orc.Tree(desc)
    level, leaf = tree.cells()
    T = np.where(leaf, 200.0, 0.0)
    em = _dust_source(orc, tree, optics, T)
    nl = len(optics.kappa_ext)
    self_abs = np.zeros((nl, tree.n_cells))
    self_emit = np.zeros((nl, tree.n_cells))
    r = orc.trace(tree, [orc._DustSource(em)], optics, 3000, seed=8, iter_=1, per_lambda=True, self_absorbed=self_abs,
                  self_emitted=self_emit)
    A = r["absorbed"]
    assert np.all(self_abs <= A * (1 + 1e-12)) and self_abs.sum() > 0
    assert np.all(self_abs <= self_emit * (1 + 1e-12))
    # each cell sends floor or ceil of E_bc / w_b packages of energy w_b
    # (Sect. 4.2), so every bin's packages carry its emission up to the
    # rounding of the cells' counts
    assert np.all(self_emit[:, ~leaf] == 0.0)
    w = em.sum(axis=1) / 3000
    for b in range(nl):
        if not w[b] > 0:          # a bin in which 200 K dust emits nothing
            assert np.all(self_emit[b] == 0.0)
            continue
        x = em[b] / w[b]
        n = np.rint(self_emit[b] / w[b])
        assert np.all(np.abs(self_emit[b] - n * w[b]) <= 1e-9 * w[b])
        assert np.all((n >= np.floor(x)) & (n <= np.ceil(x)))
        f = x - np.floor(x)
        assert abs(self_emit[b].sum() - em[b].sum()) <= 5 * w[b] * np.sqrt(np.sum(f * (1 - f))) + 1e-9 * em[b].sum()


def test_p13_weighted_temperature_solve(orc):
    """The ALI temperature solve, sum_b w_b E_b(T) = rhs: with a single
    nonzero weight it inverts one bin's Planck term in closed form,
    T = h nu / (k ln(1 + 2 h nu^3 w kappa dnu 4 pi m / (c^2 rhs))); with
    uniform weights w it is the plain solve of rhs / w."""
    desc, optics, _ = _sub_model()
    tree = orc.Tree(desc)
    level, leaf = tree.cells()
    lam = np.asarray(optics.lambda_um)
    kabs = (1 - np.asarray(optics.albedo)) * np.asarray(optics.kappa_ext)
    dnu = np.asarray(optics.dnu)
    nl, nc = lam.size, tree.n_cells
    h0 = desc.box[0] / desc.root[0]
    mass = np.asarray(desc.density) * (h0 * 0.5 ** level) ** 3
    T_true = np.where(leaf, np.random.default_rng(4).uniform(20.0, 800.0, nc), 0.0)
    H, K, CL = 6.62607015e-27, 1.380649e-16, 2.99792458e10
    b = 3
    nu = CL / (lam[b] * 1e-4)
    planck = 2 * H * nu ** 3 / CL ** 2 / np.expm1(H * nu / (K * np.where(leaf, T_true, 1e3)))
    w = np.zeros((nl, nc))
    w[b] = 0.37
    rhs = np.where(leaf, w[b] * 4 * np.pi * mass * kabs[b] * planck * dnu[b], 0.0)
    T = orc.dust_temperature_weighted(tree, rhs, w, lam, kabs, dnu, T_min=2.7, T_max=3000.0)
    np.testing.assert_allclose(T[leaf], T_true[leaf], rtol=1e-11)
    # uniform weights: the plain solve of rhs / w
    A = np.where(leaf, np.random.default_rng(5).uniform(0.1, 10.0, nc) * mass, 0.0)
    wu = np.full((nl, nc), 0.25)
    Tw = orc.dust_temperature_weighted(tree, A, wu, lam, kabs, dnu)
    Tp = orc.dust_temperature(tree, A / 0.25, lam, kabs, dnu)
    np.testing.assert_allclose(Tw[leaf], Tp[leaf], rtol=1e-11)


def test_p13_ali_sparse_packages(orc):
    """ALI (Eq. 3) with dust packages spread over cells and bins in
    proportion to the emission, so that a cell sends few or no packages in
    its weak bins.  Eight equal cells around a star, thick to their own
    emission (tau ~ 5e4 per cell at 1 um): the temperatures it settles at
    approach the well-sampled solution (ALI with 2e4 packages in every bin;
    3x more changes it by 0.5 %) as the packages grow, and stay within 12 %
    of it with 2000 packages a step.  Counting the unsampled bins as
    escaping in full (Lambda_b = 0) leaves them 20 % too cold there."""
    L = 5 * synth.AU_CM
    rho = 1e-18
    tree = orc.Tree(synth.uniform_tree((2, 2, 2), (L,) * 3, rho))
    lam = synth.log_lambda_grid(20)
    o = synth.powerlaw_dust(lam, 1e5 / (rho * L), 1.0)
    optics = synth.Optics(o.lambda_um, o.kappa_ext, np.zeros(lam.size), np.zeros(lam.size), o.dnu)
    star = synth.Source("point", bin_energy=synth.blackbody_star_bins(lam, 4000.0, 2 * synth.RSUN_CM),
                        pos=(0.5 * L,) * 3)
    kw = dict(schedule=["full"] * 25, sub_level=0, min_hits=0.0, ali=True, ali_min_packages=1, n_threads=8)
    T_ref, hist, _ = orc.lambda_subiterate(tree, star, optics, 200000, 20000, seed=3, dust_per_bin=True, **kw)
    assert hist[-1] < 0.05
    ref = T_ref.mean()
    bias = {}
    for total in (2000, 8000):
        m = [orc.lambda_subiterate(tree, star, optics, 200000, total, seed=10 + k, **kw)[0].mean() for k in range(16)]
        bias[total] = abs(np.mean(m) / ref - 1.0)
    assert bias[2000] < 0.12
    assert bias[8000] < 0.04 and bias[8000] < bias[2000]


def test_p13_ali_reaches_the_plain_fixed_point(orc):
    """ALI (Eq. 3) changes how fast the iteration gets there, not where it
    goes.  A refined cube thick to its own emission (its cells re-absorb over
    a third of what they emit): eight ALI steps end at the mass-weighted
    temperature of sixty plain Lambda steps (Eq. 2, whose fixed point the
    self-heating pin checks) to 0.2 %, where eight plain steps are still
    several times further away; per cell the two fixed points agree to the
    Monte Carlo noise that ALI's solve amplifies in such cells."""
    L = 20 * synth.AU_CM
    desc = synth.random_refined_tree((4, 4, 4), (L,) * 3, 3, 0.35, 17,
                                     rho_fn=lambda l, x, y, z: np.random.default_rng(l + 5).uniform(0.5e-18, 2e-18,
                                                                                                    x.size))
    tree = orc.Tree(desc)
    level, leaf = tree.cells()
    lam = synth.log_lambda_grid(8)
    o = synth.powerlaw_dust(lam, 200.0 / (1e-18 * L), 1.0)
    optics = synth.Optics(o.lambda_um, o.kappa_ext, np.zeros(lam.size), np.zeros(lam.size), o.dnu)
    star = synth.Source("point", bin_energy=synth.blackbody_star_bins(lam, 4000.0, 2 * synth.RSUN_CM),
                        pos=(0.47 * L, 0.52 * L, 0.49 * L))
    kw = dict(seed=6, sub_level=0, min_hits=0.0, dust_per_bin=True, n_threads=8)
    T_long, _, _ = orc.lambda_subiterate(tree, star, optics, 40000, 4000, schedule=["full"] * 60, **kw)
    T_8, _, _ = orc.lambda_subiterate(tree, star, optics, 40000, 4000, schedule=["full"] * 8, **kw)
    T_ali, _, _ = orc.lambda_subiterate(tree, star, optics, 40000, 4000, schedule=["full"] * 8, ali=True,
                                        ali_min_packages=20, **kw)
    h = (desc.box[0] / desc.root[0]) * 0.5 ** level
    mass = np.where(leaf, desc.density * h ** 3, 0.0)
    mw = lambda T: float(np.sum(mass * T) / mass.sum())
    d_ali = abs(mw(T_ali) / mw(T_long) - 1)
    d_plain = abs(mw(T_8) / mw(T_long) - 1)
    assert d_ali < 2e-3, (mw(T_ali), mw(T_long))
    assert d_plain > 3 * d_ali, (mw(T_8), mw(T_ali), mw(T_long))
    assert np.median(np.abs(T_ali[leaf] / T_long[leaf] - 1)) < 0.05
    # the diagonal of Lambda at the fixed point: the share of their emission
    # the cells re-absorb themselves
    kabs = (1 - optics.albedo) * optics.kappa_ext
    em = orc.dust_emission(tree, T_long, lam, kabs, optics.dnu)
    sa, se, sn = np.zeros_like(em), np.zeros_like(em), np.zeros(tree.n_cells)
    orc.trace(tree, [orc._DustSource(em)], optics, np.where(em.sum(axis=1) > 0, 4000, 0), seed=8, iter_=1,
              per_lambda=False, per_level=True, self_absorbed=sa, self_emitted=se, self_count=sn, n_threads=8)
    assert sa.sum() / se.sum() > 0.3, sa.sum() / se.sum()
