"""GPU tests for batched launches (many models, one persistent launch), their
CUDA-graph replay and the autotuner: a model's result is the same alone and
inside a batch."""
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


def _close(got, ref, rtol=1e-8):
    np.testing.assert_allclose(got, ref, rtol=rtol, atol=1e-9 * max(np.abs(ref).max(), 1e-300))


@pytest.fixture(scope="module")
def models():
    return synth.batch_models(n_models=6, seed=77, n_lambda=4, min_packets=2e4, max_packets=2e5, roots=(16, 32),
                              max_levels=2)


def _jobs(rt, ctx, models, precision, peel_every=0):
    grids, jobs = [], []
    for i, m in enumerate(models):
        g = rt.Grid(ctx, m.tree)
        grids.append(g)
        ab = torch.zeros((m.optics.n_lambda, g.n_cells), dtype=torch.float64, device=DEV)
        kw = dict(seed=m.seed, job=i, precision=precision, packets_per_bin=m.packets_per_bin)
        obs = img = None
        if peel_every and i % peel_every == 0:
            obs = synth.axis_observers(16, m.tree.box[0], "+z")
            img = torch.zeros((1, m.optics.n_lambda, 16, 16), dtype=torch.float64, device=DEV)
        jobs.append(rt.Job(g, m.sources, m.optics, ab, obs, img, **kw))
    return grids, jobs


def test_batch_equals_individual_fp64(rt, ctx, models):
    grids, jobs = _jobs(rt, ctx, models, 64, peel_every=2)
    leds = rt.rt_trace_batch(ctx, jobs)
    for j, led in zip(jobs, leds):
        ab = torch.zeros_like(j.absorbed)
        if j.observers is not None:
            im = torch.zeros_like(j.images)
            ref = rt.rt_peel(ctx, j.grid, j.sources, j.optics, j.observers, im, ab, **j.params)
            _close(j.images.cpu().numpy(), im.cpu().numpy())
        else:
            ref = rt.rt_trace(ctx, j.grid, j.sources, j.optics, ab, **j.params)
        _close(j.absorbed.cpu().numpy(), ab.cpu().numpy())
        for k in ("n_packets", "n_cross", "n_scatter", "n_peel_cross"):
            assert led[k] == ref[k], k
        assert led["emitted"] == pytest.approx(ref["emitted"], rel=1e-10)  # FP64 atomics, any order


def test_batch_graph_replay(rt, ctx, models):
    grids, jobs = _jobs(rt, ctx, models, 32, peel_every=3)
    b = rt.Batch(ctx, jobs)
    l1 = b.run()
    r1 = [j.absorbed.cpu().numpy().copy() for j in jobs]
    i1 = [j.images.cpu().numpy().copy() for j in jobs if j.images is not None]
    l2 = b.run()                       # outputs are zeroed inside the graph
    for j, a in zip(jobs, r1):
        _close(j.absorbed.cpu().numpy(), a)
    for j, a in zip([j for j in jobs if j.images is not None], i1):
        _close(j.images.cpu().numpy(), a)
    assert [x["n_cross"] for x in l1] == [x["n_cross"] for x in l2]
    # the graph gives what the one-shot batched launch gives
    for j in jobs:
        j.absorbed.zero_()
        if j.images is not None:
            j.images.zero_()
    rt.rt_trace_batch(ctx, jobs)
    for j, a in zip(jobs, r1):
        _close(j.absorbed.cpu().numpy(), a)
    b.close()


def test_autotune_and_persistence(rt, ctx, models, tmp_path):
    grids, jobs = _jobs(rt, ctx, models[:3], 32)
    best = rt.rt_autotune(ctx, jobs, sample_fraction=0.2)
    assert best["block_size"] in (128, 256) and best["refill_threshold"] in (2, 4, 8, 12, 16)
    assert best["crossings_per_ms"] > 0
    for j in jobs:  # the trials' accumulations were cleared
        assert float(j.absorbed.abs().sum()) == 0.0
    path = str(tmp_path / "tune.txt")
    rt.rt_tune_save(ctx, path)
    text = open(path).read()
    assert f"{best['block_size']} {best['refill_threshold']}" in text
    ctx2 = rt.Context(0)
    rt.rt_tune_load(ctx2, path)
    leds = rt.rt_trace_batch(ctx2, jobs)
    assert all(x["n_packets"] > 0 for x in leds)


def test_batched_fp64_jobs_match_oracle(rt, ctx, models, orc):
    """Inside one batched launch, FP64 jobs (with and without peel-off) give
    the oracle's absorbed energy and images for their own (seed, job) key."""
    grids, jobs = _jobs(rt, ctx, models, 64, peel_every=2)
    rt.rt_trace_batch(ctx, jobs)
    for i in (0, 1, 4):
        j, m = jobs[i], models[i]
        ref = orc.trace(orc.Tree(m.tree), m.sources, m.optics, m.packets_per_bin, seed=m.seed, job=i,
                        observers=j.observers, n_threads=8)
        _close(j.absorbed.cpu().numpy(), ref["absorbed"])
        if j.observers is not None:
            _close(j.images.cpu().numpy(), ref["images"])
