"""GPU parity for resampling at grid boundaries (Sect. 2.3, Table 1): the
CUDA tracer, whose split copies travel as records through the rounds of the
tiled tracer, against the oracle, which follows each copy after its
package.  FP64 with the same random streams: absorbed energy, images and
counters to the FP64 tolerances of the other parity tests, the same number
of copies, the primaries' own outcomes per package.  FP32: the level sums
within a few per cent of the FP64 run."""
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


def _optics(kext, albedo=0.0, g=0.0):
    return synth.Optics(lambda_um=np.array([0.55]), kappa_ext=np.array([kext]), albedo=np.array([albedo]),
                        g_hg=np.array([g]), dnu=np.ones(1))


def _nested_tree(levels=3, contrast=4.0):
    def refine(l, x, y, z, r):
        c = 2 * 2 ** l
        h = 0.75 * 2 ** l
        return (np.abs(x + 0.5 - c) < h) & (np.abs(y + 0.5 - c) < h) & (np.abs(z + 0.5 - c) < h)
    return synth.grow_tree((4, 4, 4), (4.0,) * 3, levels, lambda l, x, y, z: np.full(x.size, contrast ** l), refine)


def _case(name):
    if name == "nested_external":
        return _nested_tree(), [synth.Source("external", bin_energy=np.array([1.0]))], \
            _optics(1.0, 0.5, 0.3), None, 3000, dict(split_factor=4, rr_wmin=1e-3, rr_p=0.5), 0
    if name == "nested_point_peel":
        obs = synth.axis_observers(16, 4.0, "all6")
        return _nested_tree(), [synth.Source("point", bin_energy=np.array([1.0]), pos=(2.03, 1.96, 2.11))], \
            _optics(0.7, 0.6, 0.2), obs, 3000, dict(split_factor=2), 0
    m = synth.cloud(n_root=32, levels=2, seed=5, n_lambda=4, packets_per_bin=0, n_pix=32)
    return m.tree, m.sources, m.optics, None, 2000, dict(split_factor=4, rr_wmin=1e-3, rr_p=0.5), 8


def _run_gpu(rt, desc, sources, optics, obs, npk, precision, kw, edge=0, seed=7):
    c = rt.Context(0)
    c.set_tiles(edge)
    g = rt.Grid(c, desc)
    nl = len(optics.kappa_ext)
    ab = _zeros(nl, g.n_cells)
    log = _zeros(npk * nl * len(sources), 10)
    im = None
    if obs is not None:
        im = _zeros(obs.n_obs, nl, obs.ny, obs.nx)
        led = rt.rt_peel(c, g, sources, optics, obs, im, ab, seed=seed, precision=precision, packets_per_bin=npk,
                         packet_log=log, **kw)
    else:
        led = rt.rt_trace(c, g, sources, optics, ab, seed=seed, precision=precision, packets_per_bin=npk,
                          packet_log=log, **kw)
    out = (ab.cpu().numpy(), None if im is None else im.cpu().numpy(), log.cpu().numpy(), led)
    c.close()
    return out


@pytest.mark.parametrize("name", ["nested_external", "nested_point_peel", "cloud_tiles"])
def test_split_matches_oracle_fp64(rt, orc, name):
    desc, sources, optics, obs, npk, kw, edge = _case(name)
    ab, im, log, led = _run_gpu(rt, desc, sources, optics, obs, npk, 64, kw, edge)
    tree = orc.Tree(desc)
    ref = orc.trace(tree, sources, optics, npk, seed=7, observers=obs, record=True, n_threads=4, **kw)
    L = ref["ledger"]
    assert led["n_split_skipped"] == 0
    assert led["n_split"] == L["n_split"] and L["n_split"] > 500
    if edge:
        assert led["n_tiles"] > 1
    for k in ("n_packets", "n_cross", "n_scatter"):
        assert led[k] == L[k], k
    for k in ("emitted", "absorbed", "escaped", "rr_gain", "rr_loss"):
        assert led[k] == pytest.approx(L[k], rel=1e-9, abs=1e-12 * L["emitted"]), k
    np.testing.assert_allclose(ab, ref["absorbed"], rtol=1e-8, atol=1e-9 * np.abs(ref["absorbed"]).max())
    if obs is not None:
        np.testing.assert_allclose(im, ref["images"], rtol=1e-8, atol=1e-9 * np.abs(ref["images"]).max())
        assert led["n_peel_cross"] == L["n_peel_cross"]
    # the primaries' own paths: fate, scatterings, escaped weight
    o = ref["rec"]
    assert np.array_equal(log[:, 3], o[:, 3]) and np.array_equal(log[:, 1], o[:, 1])
    np.testing.assert_allclose(log[:, 0], o[:, 0], rtol=1e-9, atol=1e-12 * np.abs(o[:, 0]).max())
    assert abs(led["emitted"] - led["absorbed"] - led["escaped"] - led["rr_loss"] + led["rr_gain"]) \
        < 1e-10 * led["emitted"]


def test_split_tiles_equal_one_tile(rt):
    """The copies of a split stay in the tile of their package; tiled rounds
    and a single tile give the same result (FP64, same streams)."""
    desc, sources, optics, obs, npk, kw, edge = _case("cloud_tiles")
    a = _run_gpu(rt, desc, sources, optics, obs, npk, 64, kw, 0)
    b = _run_gpu(rt, desc, sources, optics, obs, npk, 64, kw, edge)
    assert a[3]["n_tiles"] == 1 and b[3]["n_tiles"] > 1
    assert a[3]["n_split"] == b[3]["n_split"]
    np.testing.assert_array_equal(a[2], b[2])
    np.testing.assert_allclose(a[0], b[0], rtol=1e-12, atol=1e-14 * np.abs(a[0]).max())


def test_split_fp32_statistical(rt, orc):
    desc, sources, optics, obs, npk, kw, edge = _case("nested_external")
    npk = 40000
    a64 = _run_gpu(rt, desc, sources, optics, obs, npk, 64, kw)
    a32 = _run_gpu(rt, desc, sources, optics, obs, npk, 32, kw)
    led = a32[3]
    assert led["n_split_skipped"] == 0
    assert abs(led["emitted"] - led["absorbed"] - led["escaped"] - led["rr_loss"] + led["rr_gain"]) \
        < 1e-5 * led["emitted"]
    assert led["n_split"] == pytest.approx(a64[3]["n_split"], rel=0.05)
    level, leaf = orc.Tree(desc).cells()  # level and leaf masks only
    for lv in (0, 1, 3):
        s = leaf & (level == lv)
        assert a32[0][0, s].sum() == pytest.approx(a64[0][0, s].sum(), rel=0.05), lv


def test_split_rejected_where_unsupported(rt):
    desc, sources, optics, obs, npk, kw, edge = _case("nested_external")
    c = rt.Context(0)
    g = rt.Grid(c, desc)
    ab = _zeros(1, g.n_cells)
    with pytest.raises(rt.RtError):
        rt.rt_trace(c, g, sources, optics, ab, seed=1, packets_per_bin=10, split_factor=4, estimator=1)
    with pytest.raises(rt.RtError):
        rt.rt_trace(c, g, sources, optics, ab, seed=1, packets_per_bin=10, split_factor=8)  # 8^3 > 256
    c.close()
