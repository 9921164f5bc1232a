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


def test_noalloc_allocates_no_device_memory(rt):
    """The entry point's one property: after the first call on the device
    (which loads the module), further calls leave the device's free memory
    unchanged."""
    ctx = rt.Context(0)
    m = synth.tiny_clump()
    grid = rt.Grid(ctx, m.tree)
    outs = [torch.zeros((1, grid.n_cells), dtype=torch.float64, device=DEV) for _ in range(3)]
    kw = dict(seed=5, precision=32, packets_per_bin=20000)
    rt.rt_trace_noalloc(grid, m.sources, m.optics, outs[0], **kw)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for o in outs[1:]:
        rt.rt_trace_noalloc(grid, m.sources, m.optics, o, **kw)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_refuses_a_capturing_stream(rt):
    ctx = rt.Context(0)
    m = synth.tiny_clump()
    grid = rt.Grid(ctx, m.tree)
    out = torch.zeros((1, grid.n_cells), dtype=torch.float64, device=DEV)
    torch.cuda.synchronize()
    s = torch.cuda.Stream(device=DEV)
    g = torch.cuda.CUDAGraph()
    code = None
    with torch.cuda.graph(g, stream=s):
        try:
            rt.rt_trace_noalloc(grid, m.sources, m.optics, out, seed=1, packets_per_bin=10, stream=s)
        except rt.RtError as e:
            code = e.code
    assert code == rt.RT_ERR_INVALID


def test_noalloc_timeout_then_complete(rt):
    """A deadline that runs out returns RT_ERR_TIMEOUT with the kernel still
    running; once the stream has drained the result is complete."""
    ctx = rt.Context(0)
    m = synth.tiny_clump()
    grid = rt.Grid(ctx, m.tree)
    kw = dict(seed=22, precision=64, per_lambda=False)
    probe = torch.zeros((1, grid.n_cells), dtype=torch.float64, device=DEV)
    npk = 20000
    for _ in range(3):  # grow the job to a few hundred ms (small launches overstate the time per package)
        led = rt.rt_trace(ctx, grid, m.sources, m.optics, probe, packets_per_bin=npk, **kw)
        if led["kernel_ms"] >= 150.0 or npk >= 2e8:
            break
        npk = int(min(2e8, npk * min(100.0, 300.0 / max(led["kernel_ms"], 0.05))))
    ref = torch.zeros_like(probe)
    led_ref = rt.rt_trace(ctx, grid, m.sources, m.optics, ref, packets_per_bin=npk, **kw)
    assert led_ref["kernel_ms"] > 20.0, led_ref["kernel_ms"]
    stream = torch.cuda.Stream(device=DEV)
    out = torch.zeros_like(ref)
    torch.cuda.synchronize()
    with pytest.raises(rt.RtError) as e:
        rt.rt_trace_noalloc(grid, m.sources, m.optics, out, packets_per_bin=npk, timeout_s=1e-4, stream=stream, **kw)
    assert e.value.code == rt.RT_ERR_TIMEOUT
    stream.synchronize()
    _close(out.cpu().numpy(), ref.cpu().numpy())
