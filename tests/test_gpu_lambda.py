"""GPU parity for the Lambda iteration (Eq. 2, Sect. 3.2) and the hit counter
that drives its stop rule."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1206_3710_gb300 import synth  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def rt():
    from paper_1206_3710_gb300 import build
    build.build()
    from paper_1206_3710_gb300 import rt as _rt
    return _rt


@pytest.fixture(scope="module")
def ctx(rt):
    return rt.Context(0)


def _star_model(tau_scale, n=8, n_lambda=12):
    L = 20 * synth.AU_CM
    rho = 1e-18
    desc = synth.random_refined_tree((n,) * 3, (L,) * 3, 1, 0.2, 3, rho_fn=lambda l, x, y, z: np.full(x.size, rho))
    lam = synth.log_lambda_grid(n_lambda)
    optics = synth.powerlaw_dust(lam, tau_scale / (rho * L), 1.0)
    star = synth.Source("point", bin_energy=synth.blackbody_star_bins(lam, 4000.0, 2 * synth.RSUN_CM),
                        pos=(0.5 * L,) * 3)
    return desc, optics, star


def test_lambda_iteration_matches_oracle_fp64(rt, ctx, orc):
    desc, optics, star = _star_model(1.0)
    g = rt.Grid(ctx, desc)
    T = torch.zeros(g.n_cells, dtype=torch.float64, device=DEV)
    npk = 3000
    res = rt.rt_lambda_iterate(ctx, g, [star], optics, T, max_iter=3, tol=0.0, min_hits=0.0,
                               dust_packets_per_bin=npk, seed=31, precision=64, packets_per_bin=npk)
    tree = orc.Tree(desc)
    T_o, hist_o = orc.lambda_iterate(tree, star, optics, npk, npk, seed=31, max_iter=3, tol=0.0, min_hits=0.0,
                                     dust_per_bin=True)
    assert res["n_iter"] == 3 and len(hist_o) == 3
    _, leaf = tree.cells()
    Tg = T.cpu().numpy()
    np.testing.assert_allclose(Tg[leaf], T_o[leaf], rtol=1e-7)
    assert np.all(Tg[~leaf] == 0)
    np.testing.assert_allclose(res["history"], hist_o, rtol=1e-4)
    # dust self-heating raised the temperatures above the star-only ones
    assert res["dust_ledger"]["emitted"] > 0


def test_hits_count_deposits(rt, ctx):
    m = synth.tiny_clump()
    g = rt.Grid(ctx, m.tree)
    ab = torch.zeros((1, g.n_cells), dtype=torch.float64, device=DEV)
    hits = torch.zeros(g.n_cells, dtype=torch.int32, device=DEV)
    led = rt.rt_trace(ctx, g, m.sources, m.optics, ab, seed=3, precision=64, packets_per_bin=20000, hits=hits)
    h = hits.cpu().numpy()
    a = ab.cpu().numpy()[0]
    np.testing.assert_array_equal(h > 0, a > 0)
    # every positive-length segment with absorption is one deposit
    assert h.sum() <= led["n_cross"] and h.sum() > 0.9 * led["n_cross"]
    with pytest.raises(rt.RtError):  # not available with peel-off
        im = torch.zeros((1, 1, 64, 64), dtype=torch.float64, device=DEV)
        rt.rt_peel(ctx, g, m.sources, m.optics, m.observers, im, ab, seed=3, packets_per_bin=10, hits=hits)


def test_lambda_iteration_small_disc_fp32(rt, ctx):
    """The disc geometry of Sect. 4.2 at reduced size: the iteration runs to
    its stop rule or cap, temperatures stay in range and the changes shrink."""
    m = synth.disc(n_root=16, max_level=6, n_lambda=12, packets=0, target_cells=3e4, max_cells=200000)
    g = rt.Grid(ctx, m.tree)
    T = torch.zeros(g.n_cells, dtype=torch.float64, device=DEV)
    res = rt.rt_lambda_iterate(ctx, g, m.sources, m.optics, T, max_iter=30, tol=1e-3, min_hits=1000,
                               dust_packets_total=400000, seed=5, precision=32, packets_total=400000,
                               rr_wmin=1e-4, rr_p=0.9)
    Tn = T.cpu().numpy()
    leaf = m.tree.refine_flags == 0
    assert np.all((Tn[leaf] >= 2.7) & (Tn[leaf] <= 3000.0))
    hist = res["history"]
    assert 1 <= res["n_iter"] <= 30
    assert res["n_iter"] == 30 or hist[-1] < 1e-3
    assert hist[-1] <= hist[0]
    L = res["source_ledger"]
    assert abs(L["emitted"] - L["absorbed"] - L["escaped"] - L["rr_loss"] + L["rr_gain"]) < 1e-4 * L["emitted"]


def test_fp32_thin_cells_take_their_deposit(rt, ctx):
    """Near-vacuum cells of the disc, whose extinction per unit length lies
    below the f32 normal range, take their deposit from the f64 density in
    the thin limit when asked (thin_f64): with the same random streams FP32
    and FP64 agree on those cells' absorbed energy; by default FP32 gives
    them nothing."""
    m = synth.disc(n_root=16, max_level=6, n_lambda=12, packets=0, target_cells=3e4, max_cells=200000)
    g = rt.Grid(ctx, m.tree)
    nl = m.optics.n_lambda
    out = {}
    for key, prec, thin in (("f32", 32, False), (32, 32, True), (64, 64, False)):
        ab = torch.zeros((nl, g.n_cells), dtype=torch.float64, device=DEV)
        rt.rt_trace(ctx, g, m.sources, m.optics, ab, seed=11, precision=prec, packets_per_bin=20000, thin_f64=thin)
        out[key] = ab.cpu().numpy()
    tree = m.tree
    h0 = tree.box[0] / tree.root[0]
    kl = m.optics.kappa_ext[:, None] * h0 * tree.density[None, :] * 0.5 ** tree.cell_levels()[None, :]
    leaf = (tree.refine_flags == 0)[None, :]
    # clearly below the f32 normal range (cells at the threshold may round
    # either way in the kernel's f32 product)
    thin = (kl < 0.5 * np.finfo(np.float32).tiny) & leaf & (out[64] > 0)
    assert thin.sum() > 50, thin.sum()
    a32, a64 = out[32][thin], out[64][thin]
    assert np.all(a32 > 0)
    rel = np.abs(a32 / a64 - 1)
    assert np.median(rel) < 1e-3 and np.quantile(rel, 0.9) < 0.05, (np.median(rel), np.quantile(rel, 0.9))
    assert np.all(out["f32"][thin] == 0)
    # elsewhere the option changes nothing
    normal = kl >= 2 * np.finfo(np.float32).tiny
    np.testing.assert_allclose(out["f32"][normal], out[32][normal], rtol=1e-12, atol=0)


# ----------------------------------------------------------------- subiterations (Sect. 3.2, App. B)

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


@pytest.mark.parametrize("per_bin", [True, False])
def test_subiterations_match_oracle_fp64(rt, ctx, orc, per_bin):
    """A schedule of full steps and subiterations below level 1, against the
    oracle's: the same temperatures after every step sequence (dust packages
    per bin, or a total that subiterations scale by the subtrees' share of
    the emission)."""
    desc, optics, star = _sub_model()
    g = rt.Grid(ctx, desc)
    T = torch.zeros(g.n_cells, dtype=torch.float64, device=DEV)
    sched = ["full", "sub", "sub", "full", "sub"]
    npk = 2000
    dkw = dict(dust_packets_per_bin=npk) if per_bin else dict(dust_packets_total=npk * 8)
    res = rt.rt_lambda_subiterate(ctx, g, [star], optics, T, sub_level=1, schedule=sched, min_hits=0.0,
                                  seed=33, precision=64, packets_per_bin=npk, **dkw)
    tree = orc.Tree(desc)
    T_o, hist_o, _ = orc.lambda_subiterate(tree, star, optics, npk, npk if per_bin else npk * 8, seed=33,
                                           schedule=sched, sub_level=1, min_hits=0.0, dust_per_bin=per_bin)
    assert res["steps"] == sched and res["n_iter"] == len(sched)
    _, leaf = tree.cells()
    Tg = T.cpu().numpy()
    np.testing.assert_allclose(Tg[leaf], T_o[leaf], rtol=1e-7)
    np.testing.assert_allclose(res["history"], hist_o, rtol=1e-4)
    assert res["dust_ledger"]["escaped"] > 0


def test_full_steps_are_the_lambda_iteration(rt, ctx):
    """Full steps only: the subiteration driver gives the temperatures of the
    plain Lambda iteration (the level arrays only split the same field)."""
    desc, optics, star = _sub_model()
    g = rt.Grid(ctx, desc)
    kw = dict(dust_packets_per_bin=3000, seed=5, precision=64, packets_per_bin=3000, min_hits=0.0)
    T1 = torch.zeros(g.n_cells, dtype=torch.float64, device=DEV)
    rt.rt_lambda_iterate(ctx, g, [star], optics, T1, max_iter=3, tol=0.0, **kw)
    T2 = torch.zeros_like(T1)
    rt.rt_lambda_subiterate(ctx, g, [star], optics, T2, sub_level=1, schedule=["full"] * 3, **kw)
    np.testing.assert_allclose(T2.cpu().numpy(), T1.cpu().numpy(), rtol=1e-10)


def test_subiterations_automatic_small_disc(rt, ctx):
    """The automatic choice (Sect. 3.3 energy balance) on a small disc: starts
    with a full step, subiterates the deep levels, returns to full steps, and
    keeps temperatures in range."""
    m = synth.disc(n_root=16, max_level=6, n_lambda=12, packets=0, target_cells=3e4, max_cells=200000)
    g = rt.Grid(ctx, m.tree)
    T = torch.zeros(g.n_cells, dtype=torch.float64, device=DEV)
    res = rt.rt_lambda_subiterate(ctx, g, m.sources, m.optics, T, sub_level=2, max_iter=12, select_frac=0.25,
                                  min_hits=1000, dust_packets_total=400000, seed=5, precision=32,
                                  packets_total=400000, rr_wmin=1e-4, rr_p=0.9)
    assert res["steps"][0] == "full" and "sub" in res["steps"]
    Tn = T.cpu().numpy()
    leaf = m.tree.refine_flags == 0
    assert np.all((Tn[leaf] >= 2.7) & (Tn[leaf] <= 3000.0))
    assert all(a >= 0 and b >= 0 for a, b in res["imbalance"])


@pytest.mark.parametrize("min_pk", [100, 3])
def test_ali_matches_oracle_fp64(rt, ctx, orc, min_pk):
    """The accelerated Lambda iteration (diagonal operator, Eq. 3) with full
    steps and subiterations, against the oracle's.  With ALI in every cell
    that sent 3 packages, most ALI cells have bins they did not sample, which
    take the opacity envelope of their sampled bins."""
    desc, optics, star = _sub_model(tau=4.0)
    g = rt.Grid(ctx, desc)
    T = torch.zeros(g.n_cells, dtype=torch.float64, device=DEV)
    sched = ["full", "sub", "full"]
    npk = 2000
    res = rt.rt_lambda_subiterate(ctx, g, [star], optics, T, sub_level=1, schedule=sched, ali=True, min_hits=0.0,
                                  dust_packets_per_bin=npk, seed=34, precision=64, packets_per_bin=npk,
                                  ali_min_packages=min_pk)
    tree = orc.Tree(desc)
    T_o, hist_o, _ = orc.lambda_subiterate(tree, star, optics, npk, npk, seed=34, schedule=sched, sub_level=1,
                                           min_hits=0.0, dust_per_bin=True, ali=True, ali_min_packages=min_pk)
    _, leaf = tree.cells()
    np.testing.assert_allclose(T.cpu().numpy()[leaf], T_o[leaf], rtol=1e-7)
    np.testing.assert_allclose(res["history"], hist_o, rtol=1e-4)


@pytest.mark.parametrize("ali", [False, True])
def test_subiterations_tiled_equal_untiled(rt, ali):
    """The level-tracking tracer in tiled rounds (its records carry the
    shallowest grid level and the ALI emission cell) gives the untiled
    temperatures (FP64, same streams; only the order of the FP64 additions
    differs)."""
    desc, optics, star = _sub_model(tau=4.0)
    res = {}
    for edge in (0, 2):
        c = rt.Context(0)
        c.set_tiles(edge)
        g = rt.Grid(c, desc)
        T = torch.zeros(g.n_cells, dtype=torch.float64, device=DEV)
        r = rt.rt_lambda_subiterate(c, g, [star], optics, T, sub_level=1, schedule=["full", "sub", "full"], ali=ali,
                                    min_hits=0.0, dust_packets_per_bin=2000, seed=35, precision=64,
                                    packets_per_bin=2000)
        res[edge] = (T.cpu().numpy(), r)
        c.close()
    assert res[2][1]["dust_ledger"]["n_tiles"] > 1
    np.testing.assert_allclose(res[2][0], res[0][0], rtol=1e-10)
