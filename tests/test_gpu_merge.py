"""GPU parity for the bottom-up construction of the hierarchical model from a
full-resolution cube (Sect. 4.1): the level-ordered description (divide
flags, densities, cells per level) equals the oracle's bit for bit; the
description builds a grid; a too-small output capacity is reported."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.merge import merge_uniform  # noqa: E402
from paper_1206_3710_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def rt():
    from paper_1206_3710_gb300 import build
    build.build()
    from paper_1206_3710_gb300 import rt as _rt
    return _rt


def _field(shape, seed, sigma=1.5):
    rng = np.random.default_rng(seed)
    from scipy.ndimage import gaussian_filter
    g = gaussian_filter(rng.normal(size=shape), 2.0, mode="wrap")
    return np.exp(sigma * g / g.std())


@pytest.mark.parametrize("case", [((4, 4, 4), 3, 0.01), ((3, 2, 5), 3, 0.02), ((16, 16, 16), 2, 0.2),
                                  ((2, 2, 2), 5, 0.004), ((4, 4, 4), 0, 0.01)])
def test_merge_matches_oracle(rt, case):
    root, L, kappa = case
    shape = (root[2] << L, root[1] << L, root[0] << L)
    rho = _field(shape, seed=sum(shape) + L)
    box = tuple(float(r) for r in root)
    ctx = rt.Context(0)
    desc = rt.rt_merge_uniform(ctx, torch.from_numpy(rho).to("cuda:0"), root, box, kappa)
    (n_ref, flags, dens), _ = merge_uniform(rho, root, box, kappa)
    assert list(desc.n_refined) == list(n_ref)
    assert np.array_equal(desc.refine_flags, flags)
    assert np.array_equal(desc.density, dens)
    g = rt.Grid(ctx, desc)  # a valid tree
    assert g.n_cells == flags.size
    ctx.close()


def test_merge_capacity_reported(rt):
    rho = _field((16, 16, 16), seed=3)
    ctx = rt.Context(0)
    with pytest.raises(rt.RtError):
        import ctypes as C
        n_ref = np.zeros(3, dtype=np.int64)
        nl, nc = C.c_int(0), C.c_int64(0)
        r = (C.c_int * 3)(4, 4, 4)
        b = (C.c_double * 3)(4.0, 4.0, 4.0)
        flags = np.zeros(10, dtype=np.uint8)
        dens = np.zeros(10)
        t = torch.from_numpy(rho).to("cuda:0")
        rc = rt.lib().rt_merge_uniform(ctx.handle, r, b, 2, t.data_ptr(), 0.05, 0.05, 30.0, 10, flags.ctypes.data,
                                       dens.ctypes.data, n_ref.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(nl),
                                       C.byref(nc), None)
        assert nc.value > 10
        rt._check(rc)
    ctx.close()
