"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

Tolerances:
  * integer work (Philox words, grid arrays, walk cell sequences): bit-exact;
  * FP64 mode with identical random streams: per-package outcomes equal to
    1e-9 relative except at boundary ties (< 1e-4 of packages), absorbed
    energy per cell and image pixels to 1e-8 relative;
  * FP32 mode: walk lengths to 1e-5 relative; absorbed energy and pixels
    within 3 sigma of the combined Monte Carlo error (a Gaussian allows
    0.27% outside; the tests allow 1%), signed mean relative deviation below
    1% over cells with >= 1e3 hits, energy balance to 1e-5.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1206_3710_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def rt():
    from paper_1206_3710_gb300 import build
    build.build()
    from paper_1206_3710_gb300 import rt as _rt
    return _rt


@pytest.fixture(scope="module")
def ctx(rt):
    return rt.Context(0)


DEV = "cuda:0"


def _zeros(*shape):
    return torch.zeros(shape, dtype=torch.float64, device=DEV)


# ----------------------------------------------------------------- Philox

def test_philox_bit_exact(rt, ctx, orc):
    rng = np.random.default_rng(0)
    n = 4096
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:16] = 0
    ctr[16:32] = 0xFFFFFFFF
    tc = torch.from_numpy(ctr.view(np.int32)).to(DEV)
    tk = torch.from_numpy(key.view(np.int32)).to(DEV)
    out = torch.zeros((n, 4), dtype=torch.int32, device=DEV)
    rt.rt_philox(ctx, tc, tk, out)
    got = out.cpu().numpy().view(np.uint32)
    for i in range(n):
        assert np.array_equal(got[i], orc.philox4x32(ctr[i], key[i])), i


# ----------------------------------------------------------------- grid build

def _expected_arrays(desc):
    flags = desc.refine_flags.astype(bool)
    n0 = int(np.prod(desc.root))
    excl = np.concatenate([[0], np.cumsum(flags)[:-1]])
    child = np.where(flags, n0 + 8 * excl, 0).astype(np.uint32)
    rho = desc.density.copy()
    off = desc.level_offsets()
    for l in range(desc.n_levels - 2, -1, -1):
        idx = np.arange(off[l], off[l + 1])
        r = idx[flags[idx]]
        rho[r] = rho[child[r][:, None] + np.arange(8)[None, :]].mean(axis=1)
    return child, rho


@pytest.mark.parametrize("seed", [1, 2])
def test_grid_build_arrays(rt, ctx, seed):
    desc = synth.random_refined_tree((5, 3, 4), (5.0, 3.0, 4.0), 3, 0.35, seed)
    g = rt.Grid(ctx, desc)
    inf = g.info
    n = desc.n_cells
    assert inf.n_cells == n and inf.n_leaves == int((desc.refine_flags == 0).sum()) and inf.depth == desc.n_levels - 1

    child, rho = _expected_arrays(desc)
    got_child = _copy_dev(inf.child, n, np.uint32)
    got_level = _copy_dev(inf.level, n, np.uint8)
    got_rho = _copy_dev(inf.density64, n, np.float64)
    got_rho32 = _copy_dev(inf.density, n, np.float32)
    got_node = _copy_dev(inf.node, n, np.uint32)
    got_coord = _copy_dev(inf.coord, n, np.uint64)
    np.testing.assert_array_equal(got_child, child)
    np.testing.assert_array_equal(got_level, desc.cell_levels())
    np.testing.assert_allclose(got_rho, rho, rtol=1e-15)
    np.testing.assert_array_equal(got_rho32, rho.astype(np.float32))
    leaf = child == 0
    np.testing.assert_array_equal(got_node[~leaf], child[~leaf] | np.uint32(0x80000000))
    scaled = (rho[leaf] / inf.rho_scale).astype(np.float32)
    np.testing.assert_array_equal(got_node[leaf].view(np.float32), scaled)
    # coordinates: cell lower corner at its level reproduces the layout
    from tests.test_oracle_geometry import leaf_boxes
    for cid, lo, size in leaf_boxes(desc):
        lev = int(round(-math.log2(size)))
        w = int(got_coord[cid])
        xyz = np.array([w & 0x1FFFFF, (w >> 21) & 0x1FFFFF, (w >> 42) & 0x1FFFFF])
        np.testing.assert_array_equal(xyz, (lo * 2 ** lev).round().astype(int))


def test_grid_set_density_equals_a_fresh_build(rt, ctx):
    """rt_grid_set_density on a grid built from density A gives, array by
    array and bit for bit, the grid rt_build_grid builds from density B (same
    tree), also from a pinned host array on a side stream; a NaN leaf
    density is refused, and a later valid call restores the grid."""
    desc = synth.random_refined_tree((5, 3, 4), (5.0, 3.0, 4.0), 3, 0.35, 1)
    rng = np.random.default_rng(4)
    dens_b = rng.lognormal(0.0, 2.0, desc.n_cells) * 1e-20
    desc_b = synth.TreeDesc(desc.root, desc.box, desc.n_refined, desc.refine_flags, dens_b)
    ref = rt.Grid(ctx, desc_b)
    n = desc.n_cells

    def arrays(g):
        inf = g.get_info()
        return (inf.rho_scale, _copy_dev(inf.density64, n, np.float64), _copy_dev(inf.density, n, np.float32),
                _copy_dev(inf.node, n, np.uint32), _copy_dev(inf.child, n, np.uint32),
                _copy_dev(inf.coord, n, np.uint64))

    want = arrays(ref)
    g = rt.Grid(ctx, desc)
    g.set_density(dens_b)
    got = arrays(g)
    assert got[0] == want[0]
    for a, b in zip(got[1:], want[1:]):
        np.testing.assert_array_equal(a, b)
    # pinned host memory, a side stream
    pin = torch.empty(n, dtype=torch.float64, pin_memory=True)
    pin.numpy()[:] = desc.density
    side = torch.cuda.Stream()
    g.set_density(pin.numpy(), stream=side)
    side.synchronize()
    fresh = arrays(rt.Grid(ctx, desc))
    got = arrays(g)
    assert got[0] == fresh[0]
    for a, b in zip(got[1:], fresh[1:]):
        np.testing.assert_array_equal(a, b)
    bad = dens_b.copy()
    bad[np.nonzero(desc.refine_flags == 0)[0][3]] = np.nan
    with pytest.raises(rt.RtError) as e:
        g.set_density(bad)
    assert e.value.code == rt.RT_ERR_INVALID
    g.set_density(dens_b)
    got = arrays(g)
    for a, b in zip(got[1:], want[1:]):
        np.testing.assert_array_equal(a, b)
    with pytest.raises(ValueError):
        g.set_density(dens_b[:-1])


def _copy_dev(ptr, count, np_dtype):
    """Copy `count` elements at a library-owned device address into numpy."""
    import ctypes
    host = np.zeros(count, dtype=np_dtype)
    torch.cuda.synchronize()
    rc = _cudart().cudaMemcpy(host.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(ptr),
                              ctypes.c_size_t(host.nbytes), 2)  # cudaMemcpyDeviceToHost
    assert rc == 0, rc
    return host


_CUDART = None


def _cudart():
    global _CUDART
    if _CUDART is None:
        import ctypes
        import glob
        import os
        cands = []
        for base in [os.path.dirname(torch.__file__)] + list(__import__("sys").path):
            cands += glob.glob(os.path.join(base, "nvidia", "cuda_runtime", "lib", "libcudart.so*"))
            cands += glob.glob(os.path.join(base, "nvidia", "cu13", "lib", "libcudart.so*"))
        cands += glob.glob("/usr/local/cuda/lib64/libcudart.so*")
        last = None
        for c in cands:
            try:
                _CUDART = ctypes.CDLL(c)
                break
            except OSError as e:  # pragma: no cover
                last = e
        if _CUDART is None:
            raise RuntimeError(f"libcudart not found: {last}")
        _CUDART.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    return _CUDART


def test_grid_rejects_invalid(rt, ctx):
    desc = synth.random_refined_tree((2, 2, 2), (2.0, 2.0, 2.0), 2, 0.5, 3)
    bad = synth.TreeDesc(desc.root, desc.box, desc.n_refined + np.array([1] + [0] * (desc.n_levels - 1)),
                         desc.refine_flags, desc.density)
    with pytest.raises(rt.RtError) as e:
        rt.Grid(ctx, bad)
    assert e.value.code == rt.RT_ERR_INVALID
    dens = desc.density.copy()
    dens[np.nonzero(desc.refine_flags == 0)[0][0]] = np.nan
    with pytest.raises(rt.RtError):
        rt.Grid(ctx, synth.TreeDesc(desc.root, desc.box, desc.n_refined, desc.refine_flags, dens))
    with pytest.raises(rt.RtError):
        rt.Grid(ctx, synth.TreeDesc(desc.root, (2.0, 2.0, 3.0), desc.n_refined, desc.refine_flags, desc.density))


# ----------------------------------------------------------------- walks

def _walk_compare(rt, ctx, orc, desc, n_rays, precision, seed, length_rtol, max_seg=None, aim=None,
                  length_atol=0.0):
    g = rt.Grid(ctx, desc)
    tree = orc.Tree(desc)
    rng = np.random.default_rng(seed)
    h0 = desc.box[0] / desc.root[0]
    o = rng.uniform(0, 1, (n_rays, 3)) * np.array(desc.box)
    d = rng.normal(size=(n_rays, 3))
    if aim is not None:   # (point, spread): rays through a small box around the point
        d = np.asarray(aim[0]) + rng.uniform(-1, 1, (n_rays, 3)) * aim[1] - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    if precision == 32:   # both sides walk the same f32-representable ray
        o = (o / h0).astype(np.float32).astype(np.float64) * h0
        o = np.minimum(o, np.array(desc.box) * (1 - 1e-7))
        d = d.astype(np.float32).astype(np.float64)
    if max_seg is None:
        max_seg = 4 * int(sum(desc.root)) * 2 ** (desc.n_levels - 1) + 16
    to = torch.from_numpy(o).to(DEV)
    td = torch.from_numpy(d).to(DEV)
    cells = torch.zeros((n_rays, max_seg), dtype=torch.int64, device=DEV)
    lens = torch.zeros((n_rays, max_seg), dtype=torch.float64, device=DEV)
    cnt = torch.zeros(n_rays, dtype=torch.int64, device=DEV)
    rt.rt_walk(ctx, g, to, td, precision, max_seg, cells, lens, cnt)
    cells, lens, cnt = cells.cpu().numpy(), lens.cpu().numpy(), cnt.cpu().numpy()
    lev_of, _ = tree.cells()
    ties = 0
    for r in range(n_rays):
        oc, ol, om = orc.walk(tree, o[r], d[r], max_seg)
        # a ray whose exit points pass within the FP32 position error of
        # another cell face may legitimately differ (tie ray)
        margin_thr = 1e-9 if precision == 64 else 3e-6 * np.arange(1, len(om) + 1)
        if np.any(om < margin_thr):
            ties += 1
            continue
        k = int(cnt[r])
        assert k == len(oc), (r, k, len(oc))
        assert np.array_equal(cells[r, :k], oc), r
        # lengths relative to the segment, with an absolute floor of the same
        # relative size of the cell (very short corner segments)
        h_leaf = h0 * 0.5 ** lev_of[oc].astype(float)
        assert np.all(np.abs(lens[r, :k] - ol) <= length_rtol * np.maximum(ol, h_leaf) + length_atol), r
    return ties


@pytest.mark.parametrize("precision,rtol", [(64, 1e-12), (32, 1e-5)])
def test_walks_tiny_grids(rt, ctx, orc, precision, rtol):
    for seed in range(4):
        desc = synth.random_refined_tree((4, 3, 4), (4.0, 3.0, 4.0), 2, 0.45, seed)
        ties = _walk_compare(rt, ctx, orc, desc, 400, precision, 50 + seed, rtol)
        assert ties <= 400 * (0 if precision == 64 else 0.02)


@pytest.mark.parametrize("precision,rtol", [(64, 1e-12), (32, 1e-5)])
def test_walks_clump_grid(rt, ctx, orc, precision, rtol):
    m = synth.tiny_clump()
    ties = _walk_compare(rt, ctx, orc, m.tree, 2000, precision, 77, rtol)
    assert ties <= 2000 * (1e-4 if precision == 64 else 0.05)


@pytest.mark.parametrize("depth", [10, 15])
def test_walks_deep_grid(rt, ctx, orc, depth):
    """Ten and fifteen refinement levels around one point.  FP64, rays aimed
    through the deepest cells: most moves out of an octet start their search
    at a stored ancestor; at fifteen levels the deepest ones lie below the
    stored path (12 levels) and start at the root cell.  FP32, rays in random
    directions (ten levels): local coordinates keep bit-exact cell sequences
    where global FP32 coordinates could not."""
    def rho_fn(l, x, y, z):
        return np.ones(x.size)

    def refine_fn(l, x, y, z, r):
        s = 2 ** l
        c = np.array([2.3, 1.7, 2.9]) * s
        return (np.abs(x + 0.5 - c[0]) < 1.5) & (np.abs(y + 0.5 - c[1]) < 1.5) & (np.abs(z + 0.5 - c[2]) < 1.5)

    desc = synth.grow_tree((4, 4, 4), (4.0,) * 3, depth, rho_fn, refine_fn)
    assert desc.n_levels == depth + 1
    # a ray crosses at most ~20 cells of each level's 6^3 refined block.
    # Lengths: the oracle's global FP64 positions (coordinates ~2 root
    # cells) carry ~1e-15 absolute error, above a relative 1e-12 of the
    # deepest cells: an absolute floor of 1e-13 h0
    ties = _walk_compare(rt, ctx, orc, desc, 300, 64, 9, 1e-12, max_seg=4096,
                         aim=((2.3, 1.7, 2.9), 2.0 ** -(depth + 1)), length_atol=1e-13)
    assert ties <= 3      # exits within 1e-9 h0 of another face: rare even in 2^-15 cells
    if depth == 10:
        ties = _walk_compare(rt, ctx, orc, desc, 300, 32, 9, 1e-5)
        assert ties <= 300 * 0.1


# ----------------------------------------------------------------- tracing

def _run_pair(rt, ctx, orc, model, npk, precision, seed, peel=True, record=True, **kw):
    g = rt.Grid(ctx, model.tree)
    tree = orc.Tree(model.tree)
    nl = model.optics.n_lambda
    per_lambda = kw.pop("per_lambda", True)
    bins = nl if per_lambda else 1
    absorbed = _zeros(bins, g.n_cells)
    n_total = npk * nl * len(model.sources)
    log = _zeros(n_total, 10) if record else None
    obs = model.observers if peel else None
    if obs is not None:
        images = _zeros(obs.n_obs, bins, obs.ny, obs.nx)
        led = rt.rt_peel(ctx, g, model.sources, model.optics, obs, images, absorbed, seed=seed, precision=precision,
                         packets_per_bin=npk, packet_log=log, per_lambda=per_lambda, **kw)
    else:
        images = None
        led = rt.rt_trace(ctx, g, model.sources, model.optics, absorbed, seed=seed, precision=precision,
                          packets_per_bin=npk, packet_log=log, per_lambda=per_lambda, **kw)
    torch.cuda.synchronize()
    ref = orc.trace(tree, model.sources, model.optics, npk, seed=seed, observers=obs, record=record,
                    validation=True, per_lambda=per_lambda, n_threads=1, **kw)
    out = dict(led=led, absorbed=absorbed.cpu().numpy(), images=None if images is None else images.cpu().numpy(),
               log=None if log is None else log.cpu().numpy(), ref=ref)
    return out


def _close(got, ref, rtol=1e-8):
    """FP64 mode: equal to rtol, with an absolute floor of 1e-9 of the largest
    value (segments that clip a cell corner have lengths that are differences
    of nearly equal coordinates, so global and leaf-local FP64 coordinates
    give them different relative rounding)."""
    np.testing.assert_allclose(got, ref, rtol=rtol, atol=1e-9 * np.abs(ref).max())


def _per_packet(out, tol=1e-9, max_div=1e-4, per_bin=None):
    """Per-package outcomes: escaped weight, scatterings, fate, exit point.
    The weight is compared to `tol` relative with an absolute floor of 1e-12
    of the largest weight of the package's wavelength bin: a package that
    absorbed an optical depth X carries the FP64 rounding of X (~1e-16 per
    segment, grown by position errors in optically thick cells) as a relative
    error of its weight e^-X, which matters only once that weight is
    negligible."""
    g, o = out["log"], out["ref"]["rec"]
    if per_bin:
        scale = np.repeat(np.abs(o[:, 0]).reshape(-1, per_bin).max(axis=1), per_bin)
    else:
        scale = np.full(o.shape[0], np.abs(o[:, 0]).max())
    same = (np.isclose(g[:, 0], o[:, 0], rtol=tol, atol=0) | (np.abs(g[:, 0] - o[:, 0]) <= 1e-12 * scale))
    same &= (g[:, 1] == o[:, 1]) & (g[:, 3] == o[:, 3])
    same &= (True
            & np.all(np.isclose(g[:, 4:7], o[:, 4:7], rtol=tol, atol=1e-6 * np.abs(o[:, 4:7]).max()), axis=1))
    frac = 1 - same.mean()
    assert frac <= max_div, (frac, np.nonzero(~same)[0][:5])
    return same


def test_fp64_clump_per_packet_and_cells(rt, ctx, orc):
    m = synth.tiny_clump()
    out = _run_pair(rt, ctx, orc, m, 100000, 64, seed=11)
    _per_packet(out)
    led, ref = out["led"], out["ref"]["ledger"]
    # the oracle adds 1e5 equal weights one after another (~n eps rounding)
    assert abs(led["emitted"] - ref["emitted"]) < 1e-10
    # energy balance: 1e5 packages summed by FP64 atomics in arbitrary order
    assert abs(led["absorbed"] + led["escaped"] - led["emitted"]) <= 1e-11
    assert led["n_cross"] == ref["n_cross"] and led["n_scatter"] == ref["n_scatter"]
    assert led["n_peel_cross"] == ref["n_peel_cross"]
    _close(out["absorbed"], out["ref"]["absorbed"])
    _close(out["images"], out["ref"]["images"])


def _statistical(gpu, ref, sumsq, hits, npk_total, min_hits=1000):
    """Independent runs of the same estimator with npk_total packages each:
    z = difference / sqrt(2 var), var from the oracle's per-element sum of
    squared package contributions (a Gaussian leaves 0.27 % beyond 3 sigma;
    1 % allowed); signed mean relative deviation below 1 % over elements with
    at least min_hits contributions."""
    var = np.maximum(sumsq - ref * ref / npk_total, 0)
    sig = np.sqrt(2 * var)
    ok = sig > 0
    z = (gpu[ok] - ref[ok]) / sig[ok]
    assert np.mean(np.abs(z) > 3) < 0.01, np.mean(np.abs(z) > 3)
    if hits is not None:
        well = hits >= min_hits
        if well.sum():
            assert abs((gpu[well] / ref[well] - 1).mean()) < 0.01


def _shared_stream_error(gpu, ref, sumsq, npk_total, hits=None):
    """FP32 against FP64 with the same random streams: only the packages whose
    paths part ways through FP32 rounding contribute to the difference, so it
    stays far below the Monte Carlo error of one run (sigma = sqrt(var)).
    Returns (max, mean) relative error over the elements with >= 1e3
    contributions (all nonzero elements when hits is None)."""
    var = np.maximum(sumsq - ref * ref / npk_total, 0)
    sig = np.sqrt(var)
    ok = sig > 0
    d = np.abs(gpu[ok] - ref[ok]) / sig[ok]
    # independent runs would leave 16 % of elements beyond 2 sigma
    assert np.mean(d > 2) < 0.01, np.mean(d > 2)
    sel = (hits >= 1000) if hits is not None else (ref != 0)
    rel = np.abs(gpu[sel] / ref[sel] - 1)
    return float(rel.max()), float(rel.mean())


def test_fp32_clump_statistical(rt, ctx, orc):
    """FP32 tracing against the FP64 oracle, per cell and per image pixel:
    within 3 sigma of an independent oracle run, and close to the oracle run
    with the same streams."""
    m = synth.tiny_clump()
    npk = 100000
    out = _run_pair(rt, ctx, orc, m, npk, 32, seed=12)
    led = out["led"]
    assert abs(led["absorbed"] + led["escaped"] - led["emitted"]) <= 1e-5 * led["emitted"]
    ref = out["ref"]
    tree = orc.Tree(m.tree)
    ind = orc.trace(tree, m.sources, m.optics, npk, seed=112, observers=m.observers, validation=True, n_threads=8)
    _statistical(out["absorbed"][0], ind["absorbed"][0], ind["sumsq"][0], ind["hits"][0], npk)
    _statistical(out["images"], ind["images"], ind["image_sumsq"], None, npk)
    # same streams: FP32 rounding changes few paths
    g, o = out["log"], ref["rec"]
    assert np.mean(g[:, 1] == o[:, 1]) > 0.95
    a_max, a_mean = _shared_stream_error(out["absorbed"][0], ref["absorbed"][0], ref["sumsq"][0], npk,
                                         ref["hits"][0])
    assert a_mean < 2e-3, (a_max, a_mean)
    i_max, i_mean = _shared_stream_error(out["images"], ref["images"], ref["image_sumsq"], npk)
    assert np.isfinite(i_max) and i_mean < 0.1, (i_max, i_mean)


def _small_cloud(n_root=32, levels=2, n_lambda=6, seed=5):
    m = synth.cloud(n_root=n_root, levels=levels, seed=seed, n_lambda=n_lambda, packets_per_bin=0, n_pix=32)
    return m


def test_fp64_cloud_external_peel(rt, ctx, orc):
    m = _small_cloud()
    out = _run_pair(rt, ctx, orc, m, 4000, 64, seed=21)
    _per_packet(out)
    _close(out["absorbed"], out["ref"]["absorbed"])
    _close(out["images"], out["ref"]["images"])
    assert out["led"]["n_peel_cross"] == out["ref"]["ledger"]["n_peel_cross"]


@pytest.mark.parametrize("precision", [64, 32])
def test_deferred_peel_equals_inline(rt, precision):
    """Peel-off deferred to the peel-off kernel, done inline in the tracer,
    and split between the two by a queue that overflows give the same images,
    absorbed energy and counters (only the order of the FP64 additions
    differs)."""
    m = _small_cloud()
    res = {}
    for name, cap in (("deferred", -1), ("inline", 0), ("mixed", 100)):
        c = rt.Context(0)
        c.set_peel_queue(cap)
        g = rt.Grid(c, m.tree)
        nl = m.optics.n_lambda
        ab = _zeros(nl, g.n_cells)
        im = _zeros(m.observers.n_obs, nl, m.observers.ny, m.observers.nx)
        led = rt.rt_peel(c, g, m.sources, m.optics, m.observers, im, ab, seed=31, precision=precision,
                         packets_per_bin=3000, rr_wmin=1e-3, rr_p=0.5)
        res[name] = (ab.cpu().numpy(), im.cpu().numpy(), led)
        c.close()
    ab0, im0, l0 = res["inline"]
    assert l0["n_peel_deferred"] == 0 and l0["n_scatter"] > 1000
    assert res["deferred"][2]["n_peel_deferred"] == l0["n_scatter"]
    assert res["mixed"][2]["n_peel_deferred"] == 100
    for name in ("deferred", "mixed"):
        ab, im, led = res[name]
        np.testing.assert_allclose(ab, ab0, rtol=1e-12, atol=1e-14 * np.abs(ab0).max())
        np.testing.assert_allclose(im, im0, rtol=1e-12, atol=1e-14 * np.abs(im0).max())
        for k in ("n_packets", "n_cross", "n_scatter", "n_peel_cross", "n_peel_out"):
            assert led[k] == l0[k], (name, k)
        for k in ("emitted", "absorbed", "escaped", "peeled", "rr_gain", "rr_loss"):
            assert led[k] == pytest.approx(l0[k], rel=1e-12), (name, k)
        assert led["peel_ms"] > 0


@pytest.mark.parametrize("case", ["cloud64_peel", "cloud32_peel", "cloud32_trace", "clump64_analog", "clump32"])
def test_tiled_equals_untiled(rt, case):
    """Tiled tracing (rounds over (bin, tile) record queues) gives every
    package the history it has untiled: identical per-package logs and
    counters, absorbed energy and images up to the order of the FP64
    additions."""
    precision = 64 if "64" in case else 32
    peel = case.endswith("peel")
    if case.startswith("cloud"):
        m, edge, kw = _small_cloud(n_root=32, levels=2, n_lambda=4), 8, dict(rr_wmin=1e-3, rr_p=0.5)
    else:
        m, edge, kw = synth.tiny_clump(), 4, {}
        if case.endswith("analog"):
            kw["estimator"] = 1
    npk = 3000
    nl = m.optics.n_lambda
    res = {}
    for e in (0, edge):
        c = rt.Context(0)
        c.set_tiles(e)
        g = rt.Grid(c, m.tree)
        ab = _zeros(nl, g.n_cells)
        log = _zeros(npk * nl * len(m.sources), 10)
        im = None
        if peel:
            obs = m.observers
            im = _zeros(obs.n_obs, nl, obs.ny, obs.nx)
            led = rt.rt_peel(c, g, m.sources, m.optics, obs, im, ab, seed=41, precision=precision,
                             packets_per_bin=npk, packet_log=log, **kw)
        else:
            led = rt.rt_trace(c, g, m.sources, m.optics, ab, seed=41, precision=precision, packets_per_bin=npk,
                              packet_log=log, **kw)
        res[e] = (ab.cpu().numpy(), None if im is None else im.cpu().numpy(), log.cpu().numpy(), led)
        c.close()
    a0, i0, l0, led0 = res[0]
    a1, i1, l1, led1 = res[edge]
    assert led0["n_cross"] > 10000
    np.testing.assert_array_equal(l1, l0)
    np.testing.assert_allclose(a1, a0, rtol=1e-12, atol=1e-14 * np.abs(a0).max())
    if peel:
        np.testing.assert_allclose(i1, i0, rtol=1e-12, atol=1e-14 * np.abs(i0).max())
    for k in ("n_packets", "n_cross", "n_scatter", "n_peel_cross", "n_peel_out", "n_killed"):
        assert led1[k] == led0[k], k
    for k in ("emitted", "absorbed", "escaped", "peeled", "rr_gain", "rr_loss"):
        assert led1[k] == pytest.approx(led0[k], rel=1e-12), k


@pytest.mark.parametrize("precision", [64, 32])
def test_shards_are_one_run(rt, ctx, precision):
    """Launches with package offsets 0 and n are, package by package, the two
    halves of one launch of 2n packages per bin (the multi-GPU sharding):
    identical histories, weights doubled exactly, mean of the shards equal to
    the single run."""
    m = _small_cloud(n_root=32, levels=2, n_lambda=3)
    g = rt.Grid(ctx, m.tree)
    nl, n = m.optics.n_lambda, 4000

    def run(npk, off):
        ab = _zeros(nl, g.n_cells)
        log = _zeros(npk * nl, 10)
        rt.rt_trace(ctx, g, m.sources, m.optics, ab, seed=12, precision=precision, packets_per_bin=npk,
                    packet_offset=off, packet_log=log, rr_wmin=1e-3, rr_p=0.5)
        return ab.cpu().numpy(), log.cpu().numpy()

    one, l1 = run(2 * n, 0)
    a, la = run(n, 0)
    b, lb = run(n, n)
    np.testing.assert_allclose(0.5 * (a + b), one, rtol=1e-12, atol=1e-14 * one.max())
    for k in range(nl):
        half = np.concatenate([la[k * n:(k + 1) * n], lb[k * n:(k + 1) * n]])
        ref = l1[k * 2 * n:(k + 1) * 2 * n]
        np.testing.assert_array_equal(half[:, 1:], ref[:, 1:])
        np.testing.assert_array_equal(half[:, 0], 2.0 * ref[:, 0])


def test_fp64_roulette_and_summed_bins(rt, ctx, orc):
    m = _small_cloud(n_root=16, levels=2, n_lambda=4)
    out = _run_pair(rt, ctx, orc, m, 3000, 64, seed=22, rr_wmin=0.3, rr_p=0.6, per_lambda=False)
    _per_packet(out)
    led = out["led"]
    assert led["rr_loss"] > 0
    lhs = led["emitted"] + led["rr_gain"]
    rhs = led["absorbed"] + led["escaped"] + led["rr_loss"]
    assert abs(lhs - rhs) <= 1e-11 * lhs
    _close(out["absorbed"], out["ref"]["absorbed"])


def test_fp64_analog(rt, ctx, orc):
    m = synth.tiny_clump()
    out = _run_pair(rt, ctx, orc, m, 20000, 64, seed=23, estimator=1)
    _per_packet(out)
    _close(out["absorbed"], out["ref"]["absorbed"])


def test_beam_and_outside_point(rt, ctx, orc):
    desc = synth.uniform_tree((4, 4, 4), (4.0,) * 3, 1.0)
    opt = synth.Optics(np.array([0.55]), np.array([0.3]), np.array([0.0]), np.array([0.0]), np.ones(1))

    class Beam:
        kind = "beam"
        pos = (0.0, 1.5, 2.5)
        dir = (1.0, 0.0, 0.0)
        bin_energy = np.array([1.0])

    m = synth.Model("beam", desc, opt, [Beam()], None, 100, 1)
    out = _run_pair(rt, ctx, orc, m, 100, 64, seed=3, peel=False)
    np.testing.assert_allclose(out["log"][:, 0], 0.01 * math.exp(-1.2), rtol=1e-12)
    far = synth.Source("point", bin_energy=np.array([1.0]), pos=(10.0, 1.0, 1.0))
    m2 = synth.Model("far", desc, opt, [far], None, 50, 1)
    out = _run_pair(rt, ctx, orc, m2, 50, 32, seed=3, peel=False)
    assert out["led"]["escaped"] == pytest.approx(1.0) and out["led"]["n_cross"] == 0


def test_zero_packets_and_empty_medium(rt, ctx, orc):
    desc = synth.uniform_tree((3, 3, 3), (3.0,) * 3, 0.0)
    opt = synth.Optics(np.array([0.55]), np.array([1.0]), np.array([0.5]), np.array([0.3]), np.ones(1))
    src = synth.Source("point", bin_energy=np.array([1.0]), pos=(1.5, 1.5, 1.5))
    g = rt.Grid(ctx, desc)
    ab = _zeros(1, g.n_cells)
    led = rt.rt_trace(ctx, g, [src], opt, ab, seed=1, packets=np.array([0]))
    assert led["n_packets"] == 0
    led = rt.rt_trace(ctx, g, [src], opt, ab, seed=1, packets_per_bin=1000)
    assert led["escaped"] == pytest.approx(1.0, rel=1e-6) and led["absorbed"] == 0 and led["n_scatter"] == 0


def test_step_limit_reports_status(rt, ctx):
    m = synth.tiny_clump()
    g = rt.Grid(ctx, m.tree)
    ab = _zeros(1, g.n_cells)
    led = rt.rt_trace(ctx, g, m.sources, m.optics, ab, seed=1, packets_per_bin=1000, step_limit=3)
    assert led["status"] == rt.RT_ERR_STEP_LIMIT and led["n_killed"] > 0
    assert abs(led["absorbed"] + led["escaped"] + led["killed"] - led["emitted"]) < 1e-5


def test_invalid_trace_arguments(rt, ctx):
    m = synth.tiny_clump()
    g = rt.Grid(ctx, m.tree)
    ab = _zeros(1, g.n_cells)
    bad = synth.Optics(m.optics.lambda_um, m.optics.kappa_ext, np.array([1.5]), m.optics.g_hg, m.optics.dnu)
    with pytest.raises(rt.RtError):
        rt.rt_trace(ctx, g, m.sources, bad, ab, seed=1, packets_per_bin=10)
    bad = synth.Optics(m.optics.lambda_um, m.optics.kappa_ext, m.optics.albedo, np.array([1.0]), m.optics.dnu)
    with pytest.raises(rt.RtError):
        rt.rt_trace(ctx, g, m.sources, bad, ab, seed=1, packets_per_bin=10)
    with pytest.raises(rt.RtError):
        rt.rt_trace(ctx, g, m.sources, m.optics, ab, seed=1, packets_per_bin=10, precision=16)
    with pytest.raises(rt.RtError):
        rt.rt_trace(ctx, g, m.sources, m.optics, ab, seed=1)


# ----------------------------------------------------------------- dust

def test_dust_temperature_parity(rt, ctx, orc):
    desc = synth.random_refined_tree((4, 4, 4), (4e16,) * 3, 2, 0.3, 8,
                                     rho_fn=lambda l, x, y, z: np.random.default_rng(l + 1).uniform(1e-22, 1e-19, x.size))
    g = rt.Grid(ctx, desc)
    tree = orc.Tree(desc)
    lam = synth.log_lambda_grid(30)
    kabs = 300.0 * (lam / 0.55) ** -1.8
    dnu = synth.bin_dnu(lam)
    rng = np.random.default_rng(4)
    A = rng.uniform(0, 1, (3, desc.n_cells)) * 10.0 ** rng.uniform(20, 34, (3, desc.n_cells))
    A[:, :5] = 0.0
    T = _zeros(desc.n_cells)
    rt.rt_dust_temperature(ctx, g, torch.from_numpy(A).to(DEV), 3, lam, kabs, dnu, T)
    To = orc.dust_temperature(tree, A.sum(axis=0), lam, kabs, dnu)
    np.testing.assert_allclose(T.cpu().numpy(), To, rtol=1e-10)
    em = _zeros(30, desc.n_cells)
    tot = rt.rt_dust_emission(ctx, g, T, lam, kabs, dnu, em)
    eo = orc.dust_emission(tree, To, lam, kabs, dnu)
    np.testing.assert_allclose(em.cpu().numpy(), eo, rtol=1e-9, atol=1e-300)
    np.testing.assert_allclose(tot, eo.sum(axis=1), rtol=1e-10)   # summation order


@pytest.mark.parametrize("n_lambda,T_min,T_max", [(3, 2.7, 3000.0), (5, 10.0, 2000.0), (64, 2.7, 3000.0)])
def test_dust_temperature_parity_ranges(rt, ctx, orc, n_lambda, T_min, T_max):
    """The temperature solve over the whole [T_min, T_max] range, with few
    wavelength bins (where one bin's Wien tail dominates E(T) at the cold
    end) and many: absorbed energies are set from temperatures drawn
    log-uniformly, plus values beyond both ends."""
    desc = synth.random_refined_tree((8, 8, 8), (4e16,) * 3, 1, 0.2, 9,
                                     rho_fn=lambda l, x, y, z: np.full(x.size, 1e-20))
    g = rt.Grid(ctx, desc)
    tree = orc.Tree(desc)
    lam = synth.log_lambda_grid(n_lambda)
    kabs = 300.0 * (lam / 0.55) ** -1.8
    dnu = synth.bin_dnu(lam)
    _, leaf = tree.cells()
    rng = np.random.default_rng(n_lambda)
    T_true = np.exp(rng.uniform(np.log(T_min) - 0.3, np.log(T_max) + 0.3, desc.n_cells))
    T_true[:4] = [T_min, T_max, T_min * (1 + 1e-9), T_max * (1 - 1e-9)]
    # A from the oracle's own emission at T_true: rho V E(T) summed over bins
    em = orc.dust_emission(tree, np.where(leaf, T_true, 0.0), lam, kabs, dnu)
    A = em.sum(axis=0)
    A[~leaf] = 0.0
    T = _zeros(desc.n_cells)
    rt.rt_dust_temperature(ctx, g, torch.from_numpy(A[None, :]).to(DEV), 1, lam, kabs, dnu, T, T_min=T_min,
                           T_max=T_max)
    To = orc.dust_temperature(tree, A, lam, kabs, dnu, T_min=T_min, T_max=T_max)
    np.testing.assert_allclose(T.cpu().numpy(), To, rtol=1e-10)
    inside = leaf & (T_true > T_min) & (T_true < T_max) & (A > 0)
    np.testing.assert_allclose(To[inside], T_true[inside], rtol=1e-9)


def test_fp64_dust_source_per_packet(rt, ctx, orc):
    L = 20 * synth.AU_CM
    desc = synth.random_refined_tree((6, 6, 6), (L,) * 3, 2, 0.3, 4,
                                     rho_fn=lambda l, x, y, z: np.random.default_rng(l + 5).uniform(1e-19, 1e-18, x.size))
    lam = synth.log_lambda_grid(8)
    # moderate optical depth: packages that scatter hundreds of times in a
    # medium whose density jumps tenfold between cells amplify FP64 rounding
    # chaotically, and per-package comparison stops being meaningful
    optics = synth.powerlaw_dust(lam, 0.3 / (1e-18 * L), 1.0)
    kabs = (1 - optics.albedo) * optics.kappa_ext
    g = rt.Grid(ctx, desc)
    tree = orc.Tree(desc)
    rng = np.random.default_rng(2)
    Tn = rng.uniform(20, 800, desc.n_cells)
    Tn[desc.refine_flags == 1] = 0
    Td = torch.from_numpy(Tn).to(DEV)
    src = rt.DustSource(Td, lam, kabs, optics.dnu)
    npk = 2000
    em = orc.dust_emission(tree, Tn, lam, kabs, optics.dnu)
    # the cells send floor or ceil of their share: the log needs room beyond
    # the budget (a short log is refused before anything runs)
    counts = orc.dust_packages(tree, em, npk, seed=5)
    total = int(counts.sum())
    ab = _zeros(len(lam), g.n_cells)
    with pytest.raises(rt.RtError) as e:
        rt.rt_trace(ctx, g, [src], optics, ab, seed=5, precision=64, packets_per_bin=npk,
                    packet_log=_zeros(total - 1, 10))
    assert e.value.code == rt.RT_ERR_INVALID
    log = _zeros(total + 100, 10)
    led = rt.rt_trace(ctx, g, [src], optics, ab, seed=5, precision=64, packets_per_bin=npk, packet_log=log)
    assert led["n_packets"] == total
    ref = orc.trace(tree, [orc._DustSource(em)], optics, npk, seed=5, record=True)
    assert ref["ledger"]["n_packets"] == total
    assert led["emitted"] == pytest.approx(ref["ledger"]["emitted"], rel=1e-10)
    g_log = log.cpu().numpy()
    assert np.all(g_log[total:] == 0)
    # per package, with each bin's largest weight as the scale of the
    # absolute floor (bins of very different weights)
    o = ref["rec"]
    seg = np.repeat(np.arange(len(lam)), counts)
    scale = np.array([np.abs(o[seg == b, 0]).max() if (seg == b).any() else 0.0 for b in range(len(lam))])[seg]
    gl = g_log[:total]
    same = np.isclose(gl[:, 0], o[:, 0], rtol=1e-9, atol=0) | (np.abs(gl[:, 0] - o[:, 0]) <= 1e-12 * scale)
    same &= (gl[:, 1] == o[:, 1]) & (gl[:, 3] == o[:, 3])
    same &= np.all(np.isclose(gl[:, 4:7], o[:, 4:7], rtol=1e-9, atol=1e-6 * np.abs(o[:, 4:7]).max()), axis=1)
    assert (~same).sum() <= max(1, int(1e-4 * total)), np.nonzero(~same)[0][:5]
    np.testing.assert_allclose(ab.cpu().numpy().sum(), ref["absorbed"].sum(), rtol=1e-6)


# ----------------------------------------------------------------- accelerated peel-off (Sect. 2.4)

_PEEL_DIRS = np.array([[0.6, 0.8, 0.0], [0.0, 0.6, -0.8], [-0.48, 0.6, 0.64], [0.0, 0.0, 1.0]])


def _peel_model(seed=8):
    root = (20, 12, 9)
    L = 20 * synth.AU_CM
    h = L / root[0]
    desc = synth.random_refined_tree(root, tuple(r * h for r in root), 2, 0.3, seed,
                                     rho_fn=lambda l, x, y, z: np.random.default_rng(l + seed).uniform(1e-19, 1e-18,
                                                                                                      x.size))
    ups = np.array([(0.0, 0.0, 1.0) if abs(d[2]) < 0.9 else (1.0, 0.0, 0.0) for d in _PEEL_DIRS])
    # the field of view holds the projected box in every direction: no
    # scattering projects outside the image
    obs = synth.Observers(dirs=_PEEL_DIRS, ups=ups, nx=24, ny=24, fov=(2 * root[0] * h, 2 * root[0] * h))
    lam = synth.log_lambda_grid(3)
    optics = synth.powerlaw_dust(lam, 2.0 / (1e-18 * L), 1.0)
    src = synth.Source("point", bin_energy=np.ones(3), pos=(7.3 * h, 5.1 * h, 4.4 * h))
    return desc, obs, optics, src


def test_peel_tables_match_oracle(rt, ctx, orc):
    """The device's extinction tables (FP64 marches from the tile centres)
    equal the oracle's, entry by entry, with partial blocks and oblique
    directions."""
    desc, obs, _, _ = _peel_model()
    g = rt.Grid(ctx, desc)
    for block, tiles in ((8, 4), (4, 8)):
        t = rt.PeelTables(ctx, g, obs, block, tiles)
        ref = orc.peel_table(orc.Tree(desc), obs, block, tiles)
        got = t.read()
        assert got.size == ref.size and np.count_nonzero(ref) > ref.size // 5
        np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-12 * ref.max())
        t.close()


def test_peel_tabulated_fp64_matches_oracle(rt, ctx, orc):
    """rt_peel_tabulated in FP64 against the oracle's accelerated peel-off:
    the same images, absorbed energy and peel-off crossings."""
    desc, obs, optics, src = _peel_model()
    g = rt.Grid(ctx, desc)
    tree = orc.Tree(desc)
    nl, npk = optics.n_lambda, 3000
    t = rt.PeelTables(ctx, g, obs, 4, 4)
    ab = _zeros(nl, g.n_cells)
    im = _zeros(obs.n_obs, nl, obs.ny, obs.nx)
    led = rt.rt_peel_tabulated(ctx, g, [src], optics, obs, t, im, ab, seed=44, precision=64, packets_per_bin=npk)
    ref = orc.trace(tree, [src], optics, npk, seed=44, observers=obs, peel_block=4, peel_tiles=4)
    exact = orc.trace(tree, [src], optics, npk, seed=44, observers=obs)
    assert led["n_peel_deferred"] == led["n_scatter"] > 0  # every scattering went through the tables
    _close(ab.cpu().numpy(), ref["absorbed"])
    _close(im.cpu().numpy(), ref["images"])
    assert led["n_peel_out"] == 0
    # segments of zero length at edge and corner crossings are not counted:
    # the two coordinate systems round a handful of them differently
    assert led["n_peel_cross"] == pytest.approx(ref["ledger"]["n_peel_cross"], rel=1e-4)
    assert led["n_peel_cross"] < 0.5 * exact["ledger"]["n_peel_cross"]
    # the approximation stays close to the exact peel-off on this model
    assert abs(im.cpu().numpy().sum() / exact["images"].sum() - 1) < 0.05


def test_peel_tabulated_rejects_other_observers(rt, ctx):
    desc, obs, optics, src = _peel_model()
    g = rt.Grid(ctx, desc)
    t = rt.PeelTables(ctx, g, obs, 4, 4)
    other = synth.Observers(dirs=obs.dirs[::-1].copy(), ups=obs.ups[::-1].copy(), nx=obs.nx, ny=obs.ny, fov=obs.fov)
    im = _zeros(obs.n_obs, optics.n_lambda, obs.ny, obs.nx)
    with pytest.raises(rt.RtError):
        rt.rt_peel_tabulated(ctx, g, [src], optics, other, t, im, None, seed=1, packets_per_bin=10)
    with pytest.raises(rt.RtError):
        rt.PeelTables(ctx, g, obs, 3, 4)
