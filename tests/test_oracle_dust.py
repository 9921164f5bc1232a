"""Pins for the oracle's dust-temperature solve and Lambda iteration
(Sect. 3.1 Eq. 2, Sect. 3.2, and the single-component equilibrium dust of
Sect. 4)."""
import math

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
    the temperatures (dust heats dust) and dT/T shrinks with each step; at
    the end the per-cell balance holds, emission(T) = absorbed."""
    desc, optics, star = _small_star_model(3.0)
    tree = orc.Tree(desc)
    kabs = (1 - optics.albedo) * optics.kappa_ext
    r = orc.trace(tree, [star], optics, 5000, seed=4, per_lambda=False)
    T0 = orc.dust_temperature(tree, r["absorbed"][0], optics.lambda_um, kabs, optics.dnu)
    T, hist = orc.lambda_iterate(tree, star, optics, 5000, 5000, seed=4, tol=1e-3, max_iter=6, min_hits=50,
                                 n_threads=4)
    assert np.median(T / T0) > 1.01
    assert hist[-1] < hist[0]
    assert len(hist) >= 2
