"""GPU parity for polychromatic packages (Sect. 2.3): the CUDA tracer against
the oracle with the same random streams (FP64): absorbed energy per bin and
cell, images, counters and per-package outcomes; FP32 against FP64 within
Monte Carlo tolerances; unsupported combinations rejected."""
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


def _zeros(*shape):
    return torch.zeros(shape, dtype=torch.float64, device=DEV)


def _model(kind):
    desc = synth.random_refined_tree((4, 4, 4), (4.0,) * 3, 2, 0.3, 5,
                                     rho_fn=lambda l, x, y, z: np.random.default_rng(l + 7).uniform(0.5, 1.5, x.size))
    n = 7
    optics = synth.Optics(lambda_um=np.linspace(0.5, 1.0, n), kappa_ext=np.linspace(0.6, 1.4, n),
                          albedo=np.linspace(0.35, 0.65, n), g_hg=np.linspace(0.1, 0.5, n), dnu=np.ones(n))
    E = np.linspace(1.0, 0.4, n)
    src = synth.Source("external", bin_energy=E) if kind == "external" else \
        synth.Source("point", bin_energy=E, pos=(2.03, 1.96, 2.11))
    return desc, [src], optics


@pytest.mark.parametrize("kind,group,peel", [("external", 4, True), ("point", 3, True), ("external", 8, False),
                                             ("point", 2, False)])
def test_poly_matches_oracle_fp64(rt, orc, kind, group, peel):
    desc, sources, optics = _model(kind)
    npk = 2000
    ctx = rt.Context(0)
    g = rt.Grid(ctx, desc)
    nl = len(optics.kappa_ext)
    ab = _zeros(nl, g.n_cells)
    n_groups = (nl + group - 1) // group
    log = _zeros(npk * n_groups, 10)
    kw = dict(seed=17, precision=64, packets_per_bin=npk, packet_log=log, poly_group=group, rr_wmin=1e-3, rr_p=0.5)
    obs = synth.axis_observers(12, 4.0, "all6") if peel else None
    if peel:
        im = _zeros(obs.n_obs, nl, obs.ny, obs.nx)
        led = rt.rt_peel(ctx, g, sources, optics, obs, im, ab, **kw)
    else:
        led = rt.rt_trace(ctx, g, sources, optics, ab, **kw)
    ref = orc.trace(orc.Tree(desc), sources, optics, npk, seed=17, observers=obs, record=True, poly_group=group,
                    rr_wmin=1e-3, rr_p=0.5, n_threads=4)
    L = ref["ledger"]
    for k in ("n_packets", "n_cross", "n_scatter", "n_peel_cross", "n_peel_out"):
        assert led[k] == L[k], k
    for k in ("emitted", "absorbed", "escaped", "rr_gain", "rr_loss", "peeled"):
        assert led[k] == pytest.approx(L[k], rel=1e-9, abs=1e-12 * L["emitted"]), k
    A = ab.cpu().numpy()
    np.testing.assert_allclose(A, ref["absorbed"], rtol=1e-8, atol=1e-9 * np.abs(ref["absorbed"]).max())
    if peel:
        I = im.cpu().numpy()
        np.testing.assert_allclose(I, ref["images"], rtol=1e-8, atol=1e-9 * np.abs(ref["images"]).max())
    lg, o = log.cpu().numpy(), ref["rec"]
    assert np.array_equal(lg[:, 1], o[:, 1]) and np.array_equal(lg[:, 3], o[:, 3])
    np.testing.assert_allclose(lg[:, 0], o[:, 0], rtol=1e-9, atol=1e-12 * np.abs(o[:, 0]).max())
    ctx.close()


def test_poly_fp32_statistical(rt):
    desc, sources, optics = _model("external")
    ctx = rt.Context(0)
    g = rt.Grid(ctx, desc)
    nl = len(optics.kappa_ext)
    res = {}
    for prec in (64, 32):
        ab = _zeros(nl, g.n_cells)
        led = rt.rt_trace(ctx, g, sources, optics, ab, seed=5, precision=prec, packets_per_bin=100000, poly_group=4)
        res[prec] = (ab.cpu().numpy(), led)
    a64, a32 = res[64][0].sum(axis=1), res[32][0].sum(axis=1)
    np.testing.assert_allclose(a32, a64, rtol=0.02)
    assert res[32][1]["n_packets"] == res[64][1]["n_packets"]
    ctx.close()


def test_poly_rejected_where_unsupported(rt):
    desc, sources, optics = _model("external")
    ctx = rt.Context(0)
    g = rt.Grid(ctx, desc)
    ab = _zeros(7, g.n_cells)
    with pytest.raises(rt.RtError):
        rt.rt_trace(ctx, g, sources, optics, ab, seed=1, packets_per_bin=10, poly_group=9)
    with pytest.raises(rt.RtError):
        rt.rt_trace(ctx, g, sources, optics, ab, seed=1, packets_per_bin=10, poly_group=4, estimator=1)
    bad = synth.Optics(lambda_um=optics.lambda_um, kappa_ext=optics.kappa_ext,
                       albedo=np.array([0.3, 0.0, 0.5, 0.5, 0.5, 0.5, 0.5]), g_hg=optics.g_hg, dnu=optics.dnu)
    with pytest.raises(rt.RtError):  # group 0's reference bin (1) does not scatter
        rt.rt_trace(ctx, g, sources, bad, ab, seed=1, packets_per_bin=10, poly_group=4)
    ctx.close()
