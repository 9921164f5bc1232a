"""GPU tests of the job server: every request's result is the same alone
and in the mix of concurrently served requests; admission holds requests
back until device memory frees up; a request that can never fit is refused."""
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


@pytest.fixture(scope="module")
def library():
    ms = [synth.tiny_clump(), synth.cloud(n_root=32, levels=2, n_lambda=6, seed=11, packets_per_bin=0, n_pix=16)]
    ms += synth.batch_models(n_models=2, seed=5, n_lambda=4, roots=(16,), max_levels=2)
    return ms


def _close(got, ref):
    np.testing.assert_allclose(got, ref, rtol=1e-8, atol=1e-9 * max(np.abs(ref).max(), 1e-300))


def _requests(library, n=14):
    rng = np.random.default_rng(4)
    reqs = []
    for i in range(n):
        mid = int(rng.integers(len(library)))
        m = library[mid]
        params = dict(seed=900 + i, job=i, precision=32, packets_per_bin=int(rng.integers(2000, 20000)),
                      rr_wmin=1e-4, rr_p=0.9)
        obs = synth.axis_observers(16, m.tree.box[0], "+z") if i % 3 == 0 else None
        reqs.append((mid, m, obs, params))
    return reqs


def test_served_results_equal_alone(rt, ctx, library):
    srv = rt.Server(ctx, hbm_budget=4 << 30, slots=2, max_batch_jobs=8, batch_window_ms=2.0)
    for mid, m in enumerate(library):
        srv.add_model(mid, m.tree)
    reqs = _requests(library)
    tickets = [srv.submit(mid, m.sources, m.optics, obs, **p) for mid, m, obs, p in reqs]
    lat = []
    for t in tickets:
        srv.wait(t)
        done, led, ms = srv.poll(t)
        assert done and led["n_packets"] > 0
        lat.append(ms)
    results = [srv.fetch(t) for t in tickets]
    assert srv.stats()["queued"] == 0
    srv.close()
    for (mid, m, obs, p), (ab, img) in zip(reqs, results):
        g = rt.Grid(ctx, m.tree)
        a = torch.zeros((m.optics.n_lambda, g.n_cells), dtype=torch.float64, device=DEV)
        if obs is not None:
            im = torch.zeros((1, m.optics.n_lambda, 16, 16), dtype=torch.float64, device=DEV)
            rt.rt_peel(ctx, g, m.sources, m.optics, obs, im, a, **p)
            _close(img, im.cpu().numpy())
        else:
            rt.rt_trace(ctx, g, m.sources, m.optics, a, **p)
        _close(ab, a.cpu().numpy())
    assert min(lat) > 0


def test_admission_waits_for_memory(rt, ctx, library):
    m = library[1]
    grid_bytes = m.tree.n_cells * 29   # density f32, child, node u32, level u8, density f64, coords u64
    acc = m.tree.n_cells * m.optics.n_lambda * 8
    # room for the grid and one request's accumulators: requests run one by one
    srv = rt.Server(ctx, hbm_budget=grid_bytes + acc + 1024, slots=2, max_batch_jobs=8, batch_window_ms=0.0)
    srv.add_model(7, m.tree)
    ts = [srv.submit(7, m.sources, m.optics, seed=i, packets_per_bin=5000, precision=32) for i in range(4)]
    st = srv.stats()
    assert st["queued"] >= 3 - st["running"]
    assert st["used_bytes"] <= grid_bytes + acc + 1024
    # results are released one by one, which admits the next request
    for t in ts:
        srv.wait(t)
        ab, _ = srv.fetch(t)
        assert ab.sum() > 0
    with pytest.raises(rt.RtError) as e:
        big = synth.axis_observers(4096, m.tree.box[0], "+z")
        srv.submit(7, m.sources, m.optics, big, seed=1, packets_per_bin=10)
    assert e.value.code == rt.RT_ERR_BUSY
    srv.close()


def test_served_fp64_request_matches_oracle(rt, ctx, library, orc):
    """A request served among others gives the oracle's absorbed energy and
    images for its (seed, job) key."""
    srv = rt.Server(ctx, hbm_budget=4 << 30, slots=2, max_batch_jobs=8, batch_window_ms=2.0)
    for mid, m in enumerate(library):
        srv.add_model(mid, m.tree)
    m = library[1]
    obs = synth.axis_observers(16, m.tree.box[0], "+z")
    p = dict(seed=77, job=5, precision=64, packets_per_bin=3000, rr_wmin=1e-3, rr_p=0.5)
    others = [srv.submit(k % len(library), library[k % len(library)].sources, library[k % len(library)].optics,
                         seed=300 + k, job=10 + k, precision=32, packets_per_bin=20000) for k in range(6)]
    t = srv.submit(1, m.sources, m.optics, obs, **p)
    srv.wait(t)
    ab, img = srv.fetch(t)
    for o in others:
        srv.wait(o)
        srv.release(o)
    srv.close()
    ref = orc.trace(orc.Tree(m.tree), m.sources, m.optics, 3000, seed=77, job=5, observers=obs, rr_wmin=1e-3,
                    rr_p=0.5, n_threads=8)
    _close(ab, ref["absorbed"])
    _close(img, ref["images"])


def test_slots_work_at_the_same_time(rt, ctx, library):
    """With two slots and one job per launch, the device-time intervals of
    launches from the two slots intersect: a request's work starts while
    another slot's launch is still on the device."""
    srv = rt.Server(ctx, hbm_budget=4 << 30, slots=2, max_batch_jobs=1, batch_window_ms=0.0)
    m = library[1]
    srv.add_model(0, m.tree)
    ts = [srv.submit(0, m.sources, m.optics, seed=500 + k, job=k, precision=32, packets_per_bin=200000)
          for k in range(12)]
    iv = []
    for t in ts:
        srv.wait(t)
        iv.append(srv.device_times(t))
        srv.release(t)
    srv.close()
    assert all(a >= 0 and b > a for a, b in iv)
    overlaps = sum(1 for i in range(len(iv)) for k in range(i + 1, len(iv))
                   if max(iv[i][0], iv[k][0]) < min(iv[i][1], iv[k][1]))
    assert overlaps >= 3, iv
