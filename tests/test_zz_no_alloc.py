"""rt_trace_noalloc: the tracer for callers that cannot let the library
allocate device memory (their memory is owned by their own pool, or they
cannot take the synchronisation of cudaMalloc).  Its scratch is a fixed
device array instead of context buffers; its results must equal rt_trace's,
call after call (the shared scratch is cleared at the start of every call).

This file is collected last so that a failure here does not stop a
first-failure run before every other test has run.
"""
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


def _close(got, ref):
    # the tolerance of the FP64 parity tests: 1e-8 relative, absolute floor
    # 1e-9 of the largest value (accumulation order of the FP64 atomics)
    np.testing.assert_allclose(got, ref, rtol=1e-8, atol=1e-9 * np.abs(ref).max())


def _check_pair(rt, ctx, model, npk, precision, seed):
    grid = rt.Grid(ctx, model.tree)
    nl = model.optics.n_lambda
    ref = torch.zeros((nl, grid.n_cells), dtype=torch.float64, device=DEV)
    kw = dict(seed=seed, precision=precision, packets_per_bin=npk, rr_wmin=1e-3, rr_p=0.5)
    led_ref = rt.rt_trace(ctx, grid, model.sources, model.optics, ref, **kw)
    ref_np = ref.cpu().numpy()
    for _ in range(2):  # two calls in a row through the C ABI
        out = torch.zeros_like(ref)
        led = rt.rt_trace_noalloc(grid, model.sources, model.optics, out, **kw)
        torch.cuda.synchronize()
        _close(out.cpu().numpy(), ref_np)
        for k in ("n_packets", "n_cross", "n_scatter", "n_killed"):
            assert led[k] == led_ref[k], k
        for k in ("emitted", "absorbed", "escaped", "rr_gain", "rr_loss"):
            assert led[k] == pytest.approx(led_ref[k], rel=1e-10, abs=1e-14 * led_ref["emitted"]), k
        assert led["status"] == led_ref["status"]


def test_noalloc_matches_rt_trace_fp64_point_source(rt):
    ctx = rt.Context(0)
    _check_pair(rt, ctx, synth.tiny_clump(), 40000, 64, seed=17)


def test_noalloc_matches_rt_trace_fp32_external_field(rt):
    ctx = rt.Context(0)
    m = synth.cloud(n_root=32, levels=2, n_lambda=6, seed=9, packets_per_bin=0, n_pix=16)
    _check_pair(rt, ctx, m, 20000, 32, seed=18)


def test_noalloc_rejects_sizes_beyond_its_scratch(rt):
    ctx = rt.Context(0)
    m = synth.tiny_clump()
    grid = rt.Grid(ctx, m.tree)
    out = torch.zeros((1, grid.n_cells), dtype=torch.float64, device=DEV)
    with pytest.raises(rt.RtError) as e:
        rt.rt_trace_noalloc(grid, m.sources * 5, m.optics, out, seed=1, packets_per_bin=10)
    assert e.value.code == rt.RT_ERR_INVALID
    T = torch.full((grid.n_cells,), 20.0, dtype=torch.float64, device=DEV)
    dust = rt.DustSource(T, m.optics.lambda_um, m.optics.kappa_ext * 0.5, m.optics.dnu)
    with pytest.raises(rt.RtError) as e:
        rt.rt_trace_noalloc(grid, [dust], m.optics, out, seed=1, packets_per_bin=10)
    assert e.value.code == rt.RT_ERR_INVALID
