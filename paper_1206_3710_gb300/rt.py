"""Thin ctypes binding of librt.so (C ABI in include/rt.h).

Argument marshalling only: every step of the transport runs in the CUDA
library.  Device buffers are torch CUDA tensors passed by pointer; streams
are torch CUDA streams.  If the compiled library is missing this module
raises at import time: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librt.so")

RT_OK, RT_ERR_INVALID, RT_ERR_OOM, RT_ERR_CUDA, RT_ERR_STEP_LIMIT, RT_ERR_TIMEOUT, RT_ERR_BUSY = 0, -1, -2, -3, -4, -5, -6
RT_SRC_POINT, RT_SRC_EXTERNAL, RT_SRC_DUST, RT_SRC_BEAM = 0, 1, 2, 3
RT_EST_CONTINUOUS, RT_EST_ANALOG = 0, 1
SOURCE_KINDS = {"point": RT_SRC_POINT, "external": RT_SRC_EXTERNAL, "dust": RT_SRC_DUST, "beam": RT_SRC_BEAM}

EXPORTED = ["rt_ctx_create", "rt_ctx_destroy", "rt_last_error", "rt_version", "rt_build_grid", "rt_grid_get_info",
            "rt_grid_free", "rt_grid_set_density", "rt_trace", "rt_peel", "rt_dust_temperature", "rt_dust_emission",
            "rt_walk",
            "rt_philox", "rt_trace_noalloc", "rt_lambda_iterate", "rt_trace_batch", "rt_batch_create",
            "rt_batch_run", "rt_batch_destroy", "rt_autotune", "rt_tune_save", "rt_tune_load", "rt_server_create",
            "rt_server_add_model", "rt_server_submit", "rt_server_poll", "rt_server_wait", "rt_server_fetch",
            "rt_server_stats", "rt_server_destroy", "rt_server_job_times", "rt_ctx_set_peel_queue", "rt_ctx_set_tiles",
            "rt_ctx_set_tile_records", "rt_l2_read_bandwidth", "rt_descent_counts",
            "rt_peel_tables_create", "rt_peel_tables_destroy", "rt_peel_tables_size", "rt_peel_tables_read",
            "rt_peel_tabulated", "rt_lambda_subiterate", "rt_merge_uniform"]


class RtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"librt error {code}: {msg}")
        self.code = code


class rt_tree_desc(C.Structure):
    _fields_ = [("root", C.c_int * 3), ("box", C.c_double * 3), ("n_levels", C.c_int),
                ("n_refined", C.POINTER(C.c_int64)), ("refine_flags", C.POINTER(C.c_uint8)),
                ("density", C.POINTER(C.c_double))]


class rt_grid_info(C.Structure):
    _fields_ = [("n_cells", C.c_int64), ("n_leaves", C.c_int64), ("depth", C.c_int), ("root", C.c_int * 3),
                ("box", C.c_double * 3), ("bytes", C.c_size_t), ("density", C.c_void_p), ("child", C.c_void_p),
                ("level", C.c_void_p), ("node", C.c_void_p), ("density64", C.c_void_p), ("coord", C.c_void_p),
                ("rho_scale", C.c_double)]


class rt_optics(C.Structure):
    _fields_ = [("n_lambda", C.c_int), ("kappa_ext", C.POINTER(C.c_double)), ("albedo", C.POINTER(C.c_double)),
                ("g_hg", C.POINTER(C.c_double))]


class rt_dust(C.Structure):
    _fields_ = [("n_lambda", C.c_int), ("lambda_um", C.POINTER(C.c_double)), ("kappa_abs", C.POINTER(C.c_double)),
                ("dnu", C.POINTER(C.c_double)), ("T_min", C.c_double), ("T_max", C.c_double)]


class rt_source(C.Structure):
    _fields_ = [("kind", C.c_int), ("pos", C.c_double * 3), ("dir", C.c_double * 3),
                ("bin_energy", C.POINTER(C.c_double)), ("T_dev", C.c_void_p), ("dust", C.POINTER(rt_dust))]


class rt_trace_params(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("job", C.c_uint32), ("iter", C.c_uint32), ("precision", C.c_int),
                ("estimator", C.c_int), ("rr_wmin", C.c_double), ("rr_p", C.c_double), ("step_limit", C.c_int64),
                ("peel_tau_max", C.c_double), ("per_lambda", C.c_int), ("packets_per_bin", C.c_int64),
                ("packets", C.POINTER(C.c_int64)), ("packets_total", C.c_int64), ("packet_log_dev", C.c_void_p),
                ("timeout_s", C.c_double), ("block_size", C.c_int), ("refill_threshold", C.c_int),
                ("blocks_per_sm", C.c_int), ("hits_dev", C.c_void_p), ("packet_offset", C.c_int64),
                ("split_factor", C.c_int), ("split_max_level", C.c_int), ("poly_group", C.c_int),
                ("packet_log_rows", C.c_int64), ("thin_f64", C.c_int)]


LEDGER_FIELDS = ["emitted", "absorbed", "escaped", "rr_gain", "rr_loss", "killed", "peeled", "n_packets", "n_cross",
                 "n_scatter", "n_peel_cross", "n_killed", "n_peel_out", "n_peel_deferred", "status", "kernel_ms",
                 "peel_ms", "n_launches", "n_tiles", "n_rounds", "n_split", "n_split_skipped"]


class rt_ledger(C.Structure):
    _fields_ = [("emitted", C.c_double), ("absorbed", C.c_double), ("escaped", C.c_double),
                ("rr_gain", C.c_double), ("rr_loss", C.c_double), ("killed", C.c_double), ("peeled", C.c_double),
                ("n_packets", C.c_uint64), ("n_cross", C.c_uint64), ("n_scatter", C.c_uint64),
                ("n_peel_cross", C.c_uint64), ("n_killed", C.c_uint64), ("n_peel_out", C.c_uint64),
                ("n_peel_deferred", C.c_uint64), ("status", C.c_int), ("kernel_ms", C.c_double),
                ("peel_ms", C.c_double), ("n_launches", C.c_int64), ("n_tiles", C.c_int32), ("n_rounds", C.c_int32),
                ("n_split", C.c_uint64), ("n_split_skipped", C.c_uint64)]

    def as_dict(self):
        return {n: getattr(self, n) for n in LEDGER_FIELDS}


class rt_lambda_params(C.Structure):
    _fields_ = [("max_iter", C.c_int), ("tol", C.c_double), ("min_hits", C.c_double),
                ("dust_packets_total", C.c_int64), ("dust_packets_per_bin", C.c_int64)]


class rt_lambda_result(C.Structure):
    _fields_ = [("n_iter", C.c_int), ("history", C.c_double * 64), ("source_ledger", rt_ledger),
                ("dust_ledger", rt_ledger), ("ms", C.c_double)]


class rt_subiter_params(C.Structure):
    _fields_ = [("sub_level", C.c_int), ("n_steps", C.c_int), ("schedule", C.POINTER(C.c_int)),
                ("select_frac", C.c_double), ("flux_frac", C.c_double), ("ali", C.c_int),
                ("ali_min_packages", C.c_int), ("ali_max_lambda", C.c_double)]


class rt_subiter_result(C.Structure):
    _fields_ = [("lambda_", rt_lambda_result), ("step_kind", C.c_int * 64), ("imbalance", (C.c_double * 2) * 64),
                ("step_ms", C.c_double * 64)]


class rt_observers(C.Structure):
    _fields_ = [("n_obs", C.c_int), ("dir", C.POINTER(C.c_double)), ("up", C.POINTER(C.c_double)),
                ("nx", C.c_int), ("ny", C.c_int), ("fov", C.c_double * 2)]


class rt_job(C.Structure):
    _fields_ = [("grid", C.c_void_p), ("n_src", C.c_int), ("src", C.POINTER(rt_source)),
                ("optics", C.POINTER(rt_optics)), ("params", C.POINTER(rt_trace_params)),
                ("obs", C.POINTER(rt_observers)), ("images_dev", C.c_void_p), ("absorbed_dev", C.c_void_p)]


class rt_server_config(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("max_slots", C.c_int), ("max_batch_jobs", C.c_int),
                ("batch_window_ms", C.c_double), ("max_batch_packets", C.c_int64)]


class rt_serve_job(C.Structure):
    _fields_ = [("model_id", C.c_uint64), ("n_src", C.c_int), ("src", C.POINTER(rt_source)),
                ("optics", C.POINTER(rt_optics)), ("params", C.POINTER(rt_trace_params)),
                ("obs", C.POINTER(rt_observers))]


class rt_tune_result(C.Structure):
    _fields_ = [("block_size", C.c_int), ("refill_threshold", C.c_int), ("blocks_per_sm", C.c_int),
                ("crossings_per_ms", C.c_double)]


_lib = None


def lib():
    """Load librt.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1206_3710_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    L.rt_ctx_create.argtypes = [C.c_int, C.POINTER(vp)]
    L.rt_ctx_destroy.argtypes = [vp]
    L.rt_ctx_destroy.restype = None
    L.rt_last_error.restype = C.c_char_p
    L.rt_last_error.argtypes = []
    L.rt_version.restype = C.c_char_p
    L.rt_version.argtypes = []
    L.rt_ctx_set_peel_queue.argtypes = [vp, C.c_int64]
    L.rt_ctx_set_tiles.argtypes = [vp, C.c_int]
    L.rt_build_grid.argtypes = [vp, C.POINTER(rt_tree_desc), C.POINTER(vp)]
    L.rt_grid_get_info.argtypes = [vp, C.POINTER(rt_grid_info)]
    L.rt_grid_free.argtypes = [vp]
    L.rt_grid_free.restype = None
    L.rt_grid_set_density.argtypes = [vp, vp, C.POINTER(C.c_double), vp]
    L.rt_trace.argtypes = [vp, vp, C.c_int, C.POINTER(rt_source), C.POINTER(rt_optics), C.POINTER(rt_trace_params),
                           vp, C.POINTER(rt_ledger), vp]
    L.rt_peel.argtypes = [vp, vp, C.c_int, C.POINTER(rt_source), C.POINTER(rt_optics), C.POINTER(rt_trace_params),
                          C.POINTER(rt_observers), vp, vp, C.POINTER(rt_ledger), vp]
    L.rt_dust_temperature.argtypes = [vp, vp, vp, C.c_int, C.POINTER(rt_dust), vp, vp]
    L.rt_peel_tables_create.argtypes = [vp, vp, C.POINTER(rt_observers), C.c_int, C.c_int, C.POINTER(vp), vp]
    L.rt_peel_tables_destroy.argtypes = [vp]
    L.rt_peel_tables_destroy.restype = None
    L.rt_peel_tables_size.argtypes = [vp]
    L.rt_peel_tables_size.restype = C.c_int64
    L.rt_peel_tables_read.argtypes = [vp, vp, C.c_int64]
    L.rt_peel_tabulated.argtypes = [vp, vp, C.c_int, C.POINTER(rt_source), C.POINTER(rt_optics),
                                    C.POINTER(rt_trace_params), C.POINTER(rt_observers), vp, vp, vp,
                                    C.POINTER(rt_ledger), vp]
    L.rt_dust_emission.argtypes = [vp, vp, vp, C.POINTER(rt_dust), vp, vp, vp]
    L.rt_walk.argtypes = [vp, vp, C.c_int64, vp, vp, C.c_int, C.c_int64, vp, vp, vp, vp]
    L.rt_merge_uniform.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_int, vp, C.c_double, C.c_double,
                                   C.c_double, C.c_int64, vp, vp, C.POINTER(C.c_int64), C.POINTER(C.c_int),
                                   C.POINTER(C.c_int64), vp]
    L.rt_philox.argtypes = [vp, C.c_int64, vp, vp, vp, vp]
    L.rt_trace_noalloc.argtypes = [vp, C.c_int, C.POINTER(rt_source), C.POINTER(rt_optics),
                                   C.POINTER(rt_trace_params), vp, C.POINTER(rt_ledger), vp]
    L.rt_lambda_iterate.argtypes = [vp, vp, C.c_int, C.POINTER(rt_source), C.POINTER(rt_optics), C.POINTER(rt_dust),
                                    C.POINTER(rt_trace_params), C.POINTER(rt_lambda_params), vp,
                                    C.POINTER(rt_lambda_result), vp]
    L.rt_trace_batch.argtypes = [vp, C.c_int, C.POINTER(rt_job), C.POINTER(rt_ledger), vp]
    L.rt_lambda_subiterate.argtypes = [vp, vp, C.c_int, C.POINTER(rt_source), C.POINTER(rt_optics),
                                       C.POINTER(rt_dust), C.POINTER(rt_trace_params), C.POINTER(rt_lambda_params),
                                       C.POINTER(rt_subiter_params), vp, C.POINTER(rt_subiter_result), vp]
    L.rt_batch_create.argtypes = [vp, C.c_int, C.POINTER(rt_job), C.POINTER(vp)]
    L.rt_batch_run.argtypes = [vp, C.POINTER(rt_ledger), C.c_double, vp]
    L.rt_batch_destroy.argtypes = [vp]
    L.rt_batch_destroy.restype = None
    L.rt_autotune.argtypes = [vp, C.c_int, C.POINTER(rt_job), C.c_double, C.POINTER(rt_tune_result)]
    L.rt_tune_save.argtypes = [vp, C.c_char_p]
    L.rt_tune_load.argtypes = [vp, C.c_char_p]
    L.rt_server_create.argtypes = [vp, C.POINTER(rt_server_config), C.POINTER(vp)]
    L.rt_server_add_model.argtypes = [vp, C.c_uint64, C.POINTER(rt_tree_desc)]
    L.rt_server_submit.argtypes = [vp, C.POINTER(rt_serve_job), C.POINTER(C.c_uint64)]
    L.rt_server_poll.argtypes = [vp, C.c_uint64, C.POINTER(C.c_int), C.POINTER(rt_ledger), C.POINTER(C.c_double)]
    L.rt_server_wait.argtypes = [vp, C.c_uint64, C.c_double]
    L.rt_server_job_times.argtypes = [vp, C.c_uint64, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.rt_l2_read_bandwidth.argtypes = [vp, vp, C.c_int64, C.c_int, C.POINTER(C.c_double), vp]
    L.rt_descent_counts.argtypes = [vp, C.POINTER(C.c_uint64), C.c_int]
    L.rt_ctx_set_tile_records.argtypes = [vp, C.c_int64]
    L.rt_server_fetch.argtypes = [vp, C.c_uint64, vp, vp]
    L.rt_server_stats.argtypes = [vp, C.POINTER(C.c_size_t), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.rt_server_destroy.argtypes = [vp]
    L.rt_server_destroy.restype = None
    for name in EXPORTED:
        if name not in ("rt_ctx_destroy", "rt_grid_free", "rt_last_error", "rt_version", "rt_batch_destroy",
                        "rt_server_destroy", "rt_peel_tables_destroy", "rt_peel_tables_size"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(rc: int, allow_step_limit: bool = False) -> int:
    if rc == RT_OK or (allow_step_limit and rc == RT_ERR_STEP_LIMIT):
        return rc
    msg = lib().rt_last_error()
    raise RtError(rc, msg.decode() if msg else "")


def _ptr(t) -> Optional[int]:
    """Device pointer of a torch tensor (or an int / None)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class _Keep:
    def __init__(self):
        self.items = []

    def arr(self, a, dtype):
        a = np.ascontiguousarray(a, dtype=dtype)
        self.items.append(a)
        return a

    def dp(self, a, dtype, ct):
        return self.arr(a, dtype).ctypes.data_as(C.POINTER(ct))


class Context:
    def __init__(self, device: int = 0):
        h = C.c_void_p()
        _check(lib().rt_ctx_create(device, C.byref(h)))
        self.handle = h
        self.device = device

    def set_peel_queue(self, max_records: int) -> None:
        """Capacity of the deferred peel-off queue in records (0: peel off
        inline in the tracer; < 0: the default)."""
        _check(lib().rt_ctx_set_peel_queue(self.handle, C.c_int64(int(max_records))))

    def set_tiles(self, tile_edge: int) -> None:
        """Tiled tracing: tile edge in root cells (a power of two), 0 off,
        < 0 automatic."""
        _check(lib().rt_ctx_set_tiles(self.handle, int(tile_edge)))

    def set_tile_records(self, max_records: int) -> None:
        """Capacity of the tiled tracer's record buffers (the emission chunk);
        <= 0: the default."""
        _check(lib().rt_ctx_set_tile_records(self.handle, C.c_int64(int(max_records))))

    def close(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.rt_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


class Grid:
    """Device grid built by rt_build_grid from a level-ordered tree desc."""

    def __init__(self, ctx: Context, desc):
        keep = _Keep()
        d = rt_tree_desc()
        d.root = (C.c_int * 3)(*desc.root)
        d.box = (C.c_double * 3)(*desc.box)
        d.n_levels = len(desc.n_refined)
        d.n_refined = keep.dp(desc.n_refined, np.int64, C.c_int64)
        d.refine_flags = keep.dp(desc.refine_flags, np.uint8, C.c_uint8)
        d.density = keep.dp(desc.density, np.float64, C.c_double)
        h = C.c_void_p()
        _check(lib().rt_build_grid(ctx.handle, C.byref(d), C.byref(h)))
        self.handle = h
        self.ctx = ctx
        self.desc = desc
        self.info = self.get_info()
        self.n_cells = int(self.info.n_cells)

    def set_density(self, density, stream=None):
        """rt_grid_set_density: new densities (host, f64, level order) for
        this grid's tree; a pinned array makes the copy asynchronous."""
        d = np.asarray(density)
        if d.dtype != np.float64 or d.ndim != 1 or d.size != self.n_cells or not d.flags["C_CONTIGUOUS"]:
            raise ValueError("set_density: a contiguous float64 array of n_cells values")
        _check(lib().rt_grid_set_density(self.ctx.handle, self.handle, d.ctypes.data_as(C.POINTER(C.c_double)),
                                         _stream(stream)))

    def get_info(self) -> rt_grid_info:
        inf = rt_grid_info()
        _check(lib().rt_grid_get_info(self.handle, C.byref(inf)))
        return inf

    def close(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.rt_grid_free(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def make_optics(optics, keep: _Keep) -> rt_optics:
    o = rt_optics()
    o.n_lambda = int(len(optics.kappa_ext))
    o.kappa_ext = keep.dp(optics.kappa_ext, np.float64, C.c_double)
    o.albedo = keep.dp(optics.albedo, np.float64, C.c_double)
    o.g_hg = keep.dp(optics.g_hg, np.float64, C.c_double)
    return o


def make_dust(lambda_um, kappa_abs, dnu, T_min, T_max, keep: _Keep) -> rt_dust:
    d = rt_dust()
    d.n_lambda = int(len(lambda_um))
    d.lambda_um = keep.dp(lambda_um, np.float64, C.c_double)
    # None: the Lambda drivers take kappa_abs = (1 - albedo) kappa_ext of the optics
    d.kappa_abs = None if kappa_abs is None else keep.dp(kappa_abs, np.float64, C.c_double)
    d.dnu = keep.dp(dnu, np.float64, C.c_double)
    d.T_min, d.T_max = float(T_min), float(T_max)
    return d


def make_sources(sources: Sequence, n_lambda: int, keep: _Keep):
    arr = (rt_source * len(sources))()
    for i, s in enumerate(sources):
        S = arr[i]
        S.kind = SOURCE_KINDS[s.kind]
        S.pos = (C.c_double * 3)(*getattr(s, "pos", (0.0, 0.0, 0.0)))
        S.dir = (C.c_double * 3)(*getattr(s, "dir", (0.0, 0.0, 1.0)))
        be = getattr(s, "bin_energy", None)
        if be is not None:
            S.bin_energy = keep.dp(be, np.float64, C.c_double)
        if s.kind == "dust":
            S.T_dev = _ptr(s.T_dev)
            d = make_dust(s.lambda_um, s.kappa_abs, s.dnu, s.T_min, s.T_max, keep)
            keep.items.append(d)
            S.dust = C.pointer(d)
    return arr


def make_params(keep: _Keep, *, seed: int, job: int = 0, iter_: int = 0, precision: int = 32,
                estimator: int = RT_EST_CONTINUOUS, rr_wmin: float = 0.0, rr_p: float = 0.9, step_limit: int = 0,
                peel_tau_max: float = 0.0, per_lambda: bool = True, packets_per_bin: int = 0, packets=None,
                packets_total: int = 0, packet_log=None, timeout_s: float = 0.0, block_size: int = 0,
                refill_threshold: int = 0, blocks_per_sm: int = 0, hits=None,
                packet_offset: int = 0, split_factor: int = 1, split_max_level: int = -1,
                poly_group: int = 1, thin_f64: bool = False) -> rt_trace_params:
    p = rt_trace_params()
    p.seed, p.job, p.iter = int(seed), int(job), int(iter_)
    p.precision, p.estimator = int(precision), int(estimator)
    p.rr_wmin, p.rr_p, p.step_limit = float(rr_wmin), float(rr_p), int(step_limit)
    p.peel_tau_max, p.per_lambda = float(peel_tau_max), int(bool(per_lambda))
    p.packets_per_bin, p.packets_total = int(packets_per_bin), int(packets_total)
    if packets is not None:
        p.packets = keep.dp(np.asarray(packets).ravel(), np.int64, C.c_int64)
    p.packet_log_dev = _ptr(packet_log)
    p.packet_log_rows = 0 if packet_log is None else int(packet_log.shape[0])
    p.timeout_s = float(timeout_s)
    p.block_size, p.refill_threshold, p.blocks_per_sm = int(block_size), int(refill_threshold), int(blocks_per_sm)
    p.hits_dev = _ptr(hits)
    p.packet_offset = int(packet_offset)
    p.split_factor, p.split_max_level = int(split_factor), int(split_max_level)
    p.thin_f64 = int(bool(thin_f64))
    p.poly_group = int(poly_group)
    return p


def make_observers(obs, keep: _Keep) -> rt_observers:
    o = rt_observers()
    o.n_obs = int(obs.dirs.shape[0])
    o.dir = keep.dp(obs.dirs, np.float64, C.c_double)
    o.up = keep.dp(obs.ups, np.float64, C.c_double)
    o.nx, o.ny = int(obs.nx), int(obs.ny)
    o.fov = (C.c_double * 2)(*obs.fov)
    return o


def rt_trace(ctx: Context, grid: Grid, sources, optics, absorbed, stream=None, **params) -> dict:
    keep = _Keep()
    src = make_sources(sources, len(optics.kappa_ext), keep)
    op = make_optics(optics, keep)
    prm = make_params(keep, **params)
    led = rt_ledger()
    rc = lib().rt_trace(ctx.handle, grid.handle, len(sources), src, C.byref(op), C.byref(prm), _ptr(absorbed),
                        C.byref(led), _stream(stream))
    _check(rc, allow_step_limit=True)
    return led.as_dict()


def rt_trace_noalloc(grid: Grid, sources, optics, absorbed, stream=None, **params) -> dict:
    """Allocation-free variant of rt_trace (scratch in a static device array)."""
    keep = _Keep()
    src = make_sources(sources, len(optics.kappa_ext), keep)
    op = make_optics(optics, keep)
    prm = make_params(keep, **params)
    led = rt_ledger()
    rc = lib().rt_trace_noalloc(grid.handle, len(sources), src, C.byref(op), C.byref(prm), _ptr(absorbed),
                                C.byref(led), _stream(stream))
    _check(rc, allow_step_limit=True)
    return led.as_dict()


def rt_peel(ctx: Context, grid: Grid, sources, optics, observers, images, absorbed=None, stream=None,
            **params) -> dict:
    keep = _Keep()
    src = make_sources(sources, len(optics.kappa_ext), keep)
    op = make_optics(optics, keep)
    prm = make_params(keep, **params)
    ob = make_observers(observers, keep)
    led = rt_ledger()
    rc = lib().rt_peel(ctx.handle, grid.handle, len(sources), src, C.byref(op), C.byref(prm), C.byref(ob),
                       _ptr(images), _ptr(absorbed), C.byref(led), _stream(stream))
    _check(rc, allow_step_limit=True)
    return led.as_dict()


class PeelTables:
    """Extinction tables of the accelerated peel-off (Sect. 2.4) for one grid
    and observer set (device memory owned by the library)."""

    def __init__(self, ctx: Context, grid: Grid, observers, block_edge: int, tiles_per_edge: int, stream=None):
        keep = _Keep()
        ob = make_observers(observers, keep)
        h = C.c_void_p()
        _check(lib().rt_peel_tables_create(ctx.handle, grid.handle, C.byref(ob), int(block_edge),
                                           int(tiles_per_edge), C.byref(h), _stream(stream)))
        self.handle, self.grid, self.observers = h, grid, observers

    @property
    def size(self) -> int:
        return int(lib().rt_peel_tables_size(self.handle))

    def read(self) -> np.ndarray:
        out = np.zeros(max(self.size, 1))
        _check(lib().rt_peel_tables_read(self.handle, out.ctypes.data_as(C.c_void_p), C.c_int64(out.size)))
        return out[:self.size]

    def close(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.rt_peel_tables_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def rt_peel_tabulated(ctx: Context, grid: Grid, sources, optics, observers, tables: PeelTables, images,
                      absorbed=None, stream=None, **params) -> dict:
    keep = _Keep()
    src = make_sources(sources, len(optics.kappa_ext), keep)
    op = make_optics(optics, keep)
    prm = make_params(keep, **params)
    ob = make_observers(observers, keep)
    led = rt_ledger()
    rc = lib().rt_peel_tabulated(ctx.handle, grid.handle, len(sources), src, C.byref(op), C.byref(prm), C.byref(ob),
                                 tables.handle, _ptr(images), _ptr(absorbed), C.byref(led), _stream(stream))
    _check(rc, allow_step_limit=True)
    return led.as_dict()


def rt_dust_temperature(ctx: Context, grid: Grid, absorbed, n_bins: int, lambda_um, kappa_abs, dnu, T_out,
                        T_min: float = 2.7, T_max: float = 3000.0, stream=None) -> None:
    keep = _Keep()
    d = make_dust(lambda_um, kappa_abs, dnu, T_min, T_max, keep)
    _check(lib().rt_dust_temperature(ctx.handle, grid.handle, _ptr(absorbed), int(n_bins), C.byref(d), _ptr(T_out),
                                     _stream(stream)))


def rt_dust_emission(ctx: Context, grid: Grid, T, lambda_um, kappa_abs, dnu, emission, stream=None) -> np.ndarray:
    keep = _Keep()
    d = make_dust(lambda_um, kappa_abs, dnu, 2.7, 3000.0, keep)
    tot = np.zeros(len(lambda_um))
    _check(lib().rt_dust_emission(ctx.handle, grid.handle, _ptr(T), C.byref(d), _ptr(emission),
                                  tot.ctypes.data_as(C.c_void_p), _stream(stream)))
    return tot


def rt_lambda_iterate(ctx: Context, grid: Grid, sources, optics, T_out, *, max_iter: int = 30, tol: float = 1e-3,
                      min_hits: float = 1000.0, dust_packets_total: int = 0, dust_packets_per_bin: int = 0,
                      T_min: float = 2.7, T_max: float = 3000.0, stream=None, **params) -> dict:
    """Lambda iteration (Eq. 2) on the device; returns iterations, history and ledgers."""
    keep = _Keep()
    src = make_sources(sources, len(optics.kappa_ext), keep)
    op = make_optics(optics, keep)
    du = make_dust(optics.lambda_um, None, optics.dnu, T_min, T_max, keep)
    prm = make_params(keep, **params)
    lp = rt_lambda_params(max_iter=int(max_iter), tol=float(tol), min_hits=float(min_hits),
                          dust_packets_total=int(dust_packets_total), dust_packets_per_bin=int(dust_packets_per_bin))
    res = rt_lambda_result()
    _check(lib().rt_lambda_iterate(ctx.handle, grid.handle, len(sources), src, C.byref(op), C.byref(du), C.byref(prm),
                                   C.byref(lp), _ptr(T_out), C.byref(res), _stream(stream)))
    return dict(n_iter=res.n_iter, history=[res.history[i] for i in range(res.n_iter)],
                source_ledger=res.source_ledger.as_dict(), dust_ledger=res.dust_ledger.as_dict(), ms=res.ms)


def rt_lambda_subiterate(ctx: Context, grid: Grid, sources, optics, T_out, *, sub_level: int, schedule=None,
                         max_iter: int = 30, select_frac: float = 0.25, flux_frac: float = 0.05,
                         ali: bool = False, ali_min_packages: int = 100, ali_max_lambda: float = 0.999,
                         tol: float = 0.0,
                         min_hits: float = 1000.0,
                         dust_packets_total: int = 0, dust_packets_per_bin: int = 0, T_min: float = 2.7,
                         T_max: float = 3000.0, stream=None, **params) -> dict:
    """Lambda iteration with subiterations (Sect. 3.2, App. B).  ``schedule``:
    a list of "full" / "sub" steps, or None for the automatic choice over
    ``max_iter`` steps."""
    keep = _Keep()
    src = make_sources(sources, len(optics.kappa_ext), keep)
    op = make_optics(optics, keep)
    du = make_dust(optics.lambda_um, None, optics.dnu, T_min, T_max, keep)
    prm = make_params(keep, **params)
    lp = rt_lambda_params(max_iter=int(max_iter), tol=float(tol), min_hits=float(min_hits),
                          dust_packets_total=int(dust_packets_total), dust_packets_per_bin=int(dust_packets_per_bin))
    sp = rt_subiter_params(sub_level=int(sub_level), n_steps=0, select_frac=float(select_frac),
                           flux_frac=float(flux_frac), ali=int(bool(ali)),
                           ali_min_packages=int(ali_min_packages), ali_max_lambda=float(ali_max_lambda))
    if schedule is not None:
        kinds = np.array([{"full": 0, "sub": 1}[k] for k in schedule], dtype=np.int32)
        sp.n_steps = len(kinds)
        sp.schedule = keep.dp(kinds, np.int32, C.c_int)
    res = rt_subiter_result()
    _check(lib().rt_lambda_subiterate(ctx.handle, grid.handle, len(sources), src, C.byref(op), C.byref(du),
                                      C.byref(prm), C.byref(lp), C.byref(sp), _ptr(T_out), C.byref(res),
                                      _stream(stream)))
    n = res.lambda_.n_iter
    return dict(n_iter=n, history=[res.lambda_.history[i] for i in range(n)],
                steps=["sub" if res.step_kind[i] else "full" for i in range(n)],
                imbalance=[(res.imbalance[i][0], res.imbalance[i][1]) for i in range(n)],
                step_ms=[res.step_ms[i] for i in range(n)], source_ledger=res.lambda_.source_ledger.as_dict(),
                dust_ledger=res.lambda_.dust_ledger.as_dict(), ms=res.lambda_.ms)


def rt_walk(ctx: Context, grid: Grid, origins, dirs, precision: int, max_seg: int, cells, lengths, counts,
            stream=None) -> None:
    n = int(origins.shape[0])
    _check(lib().rt_walk(ctx.handle, grid.handle, n, _ptr(origins), _ptr(dirs), int(precision), int(max_seg),
                         _ptr(cells), _ptr(lengths), _ptr(counts), _stream(stream)))


def rt_merge_uniform(ctx: Context, rho, root, box, kappa: float, tau_max: float = 0.05, contrast_max: float = 30.0,
                     stream=None):
    """Hierarchical model from a full-resolution cube (Sect. 4.1).  ``rho``:
    device f64 tensor [nz][ny][nx] (x fastest) with root * 2^L cells per
    axis.  Returns a tree description for ``Grid``."""
    from . import synth
    nz, ny, nx = (int(v) for v in rho.shape)
    L = 0
    while (int(root[0]) << L) < nx:
        L += 1
    cap = sum(int(np.prod(root)) << (3 * l) for l in range(L + 1))
    flags = np.zeros(cap, dtype=np.uint8)
    dens = np.zeros(cap, dtype=np.float64)
    n_ref = np.zeros(L + 1, dtype=np.int64)
    n_lev = C.c_int(0)
    n_cells = C.c_int64(0)
    r = (C.c_int * 3)(*[int(v) for v in root])
    b = (C.c_double * 3)(*[float(v) for v in box])
    _check(lib().rt_merge_uniform(ctx.handle, r, b, L, _ptr(rho), float(kappa), float(tau_max), float(contrast_max),
                                  cap, flags.ctypes.data, dens.ctypes.data,
                                  n_ref.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(n_lev), C.byref(n_cells),
                                  _stream(stream)))
    n = int(n_cells.value)
    return synth.TreeDesc(root=tuple(int(v) for v in root), box=tuple(float(v) for v in box),
                          n_refined=n_ref[: n_lev.value].copy(), refine_flags=flags[:n].copy(), density=dens[:n].copy())


def rt_l2_read_bandwidth(ctx: Context, buf, reps: int = 40, stream=None) -> float:
    """L2 read bandwidth (GB/s) over a zeroed device tensor that fits in L2."""
    gbs = C.c_double()
    _check(lib().rt_l2_read_bandwidth(ctx.handle, _ptr(buf), C.c_int64(buf.numel() * buf.element_size()),
                                      int(reps), C.byref(gbs), _stream(stream)))
    return gbs.value


def rt_descent_counts(ctx: Context, reset: bool = True):
    """(tracer, peel-off) node descents since the last reset; builds
    compiled with RT_COUNT_DESCENTS=1 only."""
    out = (C.c_uint64 * 2)()
    _check(lib().rt_descent_counts(ctx.handle, out, int(bool(reset))))
    return int(out[0]), int(out[1])


def rt_philox(ctx: Context, ctr, key, out, stream=None) -> None:
    n = int(ctr.shape[0])
    _check(lib().rt_philox(ctx.handle, n, _ptr(ctr), _ptr(key), _ptr(out), _stream(stream)))


class DustSource:
    """Thermal dust emission from device temperatures (rt_source kind dust)."""
    kind = "dust"

    def __init__(self, T_dev, lambda_um, kappa_abs, dnu, T_min=2.7, T_max=3000.0):
        self.T_dev, self.lambda_um, self.kappa_abs, self.dnu = T_dev, lambda_um, kappa_abs, dnu
        self.T_min, self.T_max = T_min, T_max
        self.bin_energy = None


class Job:
    """One model of a batched launch (the arguments of rt_trace / rt_peel)."""

    def __init__(self, grid: Grid, sources, optics, absorbed=None, observers=None, images=None, **params):
        self.grid, self.sources, self.optics, self.absorbed = grid, sources, optics, absorbed
        self.observers, self.images, self.params = observers, images, params


def _jobs_array(jobs, keep: _Keep):
    arr = (rt_job * len(jobs))()
    for i, j in enumerate(jobs):
        J = arr[i]
        J.grid = j.grid.handle
        J.n_src = len(j.sources)
        src = make_sources(j.sources, len(j.optics.kappa_ext), keep)
        op = make_optics(j.optics, keep)
        prm = make_params(keep, **j.params)
        keep.items += [src, op, prm]
        J.src = C.cast(src, C.POINTER(rt_source))
        J.optics = C.pointer(op)
        J.params = C.pointer(prm)
        if j.observers is not None:
            ob = make_observers(j.observers, keep)
            keep.items.append(ob)
            J.obs = C.pointer(ob)
        J.images_dev = _ptr(j.images)
        J.absorbed_dev = _ptr(j.absorbed)
    return arr


def rt_trace_batch(ctx: Context, jobs, stream=None):
    """All jobs in one persistent launch; returns one ledger per job."""
    keep = _Keep()
    arr = _jobs_array(jobs, keep)
    leds = (rt_ledger * len(jobs))()
    rc = lib().rt_trace_batch(ctx.handle, len(jobs), arr, leds, _stream(stream))
    _check(rc, allow_step_limit=True)
    return [leds[i].as_dict() for i in range(len(jobs))]


class Batch:
    """A batch whose launch is captured once in a CUDA graph and replayed."""

    def __init__(self, ctx: Context, jobs):
        keep = _Keep()
        arr = _jobs_array(jobs, keep)
        h = C.c_void_p()
        _check(lib().rt_batch_create(ctx.handle, len(jobs), arr, C.byref(h)))
        self.handle, self.n, self.ctx, self.jobs = h, len(jobs), ctx, jobs

    def run(self, timeout_s: float = 0.0, stream=None):
        leds = (rt_ledger * self.n)()
        _check(lib().rt_batch_run(self.handle, leds, float(timeout_s), _stream(stream)), allow_step_limit=True)
        return [leds[i].as_dict() for i in range(self.n)]

    def close(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.rt_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def rt_autotune(ctx: Context, jobs, sample_fraction: float = 0.05) -> dict:
    keep = _Keep()
    arr = _jobs_array(jobs, keep)
    res = rt_tune_result()
    _check(lib().rt_autotune(ctx.handle, len(jobs), arr, float(sample_fraction), C.byref(res)))
    return dict(block_size=res.block_size, refill_threshold=res.refill_threshold, blocks_per_sm=res.blocks_per_sm,
                crossings_per_ms=res.crossings_per_ms)


def rt_tune_save(ctx: Context, path: str) -> None:
    _check(lib().rt_tune_save(ctx.handle, path.encode()))


def rt_tune_load(ctx: Context, path: str) -> None:
    _check(lib().rt_tune_load(ctx.handle, path.encode()))


def _tree_struct(desc, keep: _Keep) -> rt_tree_desc:
    d = rt_tree_desc()
    d.root = (C.c_int * 3)(*desc.root)
    d.box = (C.c_double * 3)(*desc.box)
    d.n_levels = len(desc.n_refined)
    d.n_refined = keep.dp(desc.n_refined, np.int64, C.c_int64)
    d.refine_flags = keep.dp(desc.refine_flags, np.uint8, C.c_uint8)
    d.density = keep.dp(desc.density, np.float64, C.c_double)
    return d


class Server:
    """Job server: resident grids, admission by device-memory footprint,
    continuous batching over `slots` streams (rt_server_* in librt)."""

    def __init__(self, ctx: Context, hbm_budget: int, slots: int = 2, max_batch_jobs: int = 64,
                 batch_window_ms: float = 1.0, max_batch_packets: int = 0):
        cfg = rt_server_config(hbm_budget=int(hbm_budget), max_slots=int(slots), max_batch_jobs=int(max_batch_jobs),
                               batch_window_ms=float(batch_window_ms), max_batch_packets=int(max_batch_packets))
        h = C.c_void_p()
        _check(lib().rt_server_create(ctx.handle, C.byref(cfg), C.byref(h)))
        self.handle, self.ctx = h, ctx
        self.shapes = {}
        self.cells = {}

    def add_model(self, model_id: int, desc) -> None:
        keep = _Keep()
        d = _tree_struct(desc, keep)
        _check(lib().rt_server_add_model(self.handle, int(model_id), C.byref(d)))
        self.cells[int(model_id)] = int(desc.n_cells)

    def submit(self, model_id: int, sources, optics, observers=None, **params) -> int:
        keep = _Keep()
        src = make_sources(sources, len(optics.kappa_ext), keep)
        op = make_optics(optics, keep)
        prm = make_params(keep, **params)
        j = rt_serve_job(model_id=int(model_id), n_src=len(sources))
        j.src = C.cast(src, C.POINTER(rt_source))
        j.optics = C.pointer(op)
        j.params = C.pointer(prm)
        if observers is not None:
            ob = make_observers(observers, keep)
            keep.items.append(ob)
            j.obs = C.pointer(ob)
        t = C.c_uint64()
        _check(lib().rt_server_submit(self.handle, C.byref(j), C.byref(t)))
        bins = len(optics.kappa_ext) if params.get("per_lambda", True) else 1
        img = None if observers is None else (observers.n_obs, bins, observers.ny, observers.nx)
        self.shapes[t.value] = ((bins, self.cells[int(model_id)]), img)
        return t.value

    def device_times(self, ticket: int):
        """(start, end) in ms of device time of the launch the request ran in."""
        a, b = C.c_double(), C.c_double()
        _check(lib().rt_server_job_times(self.handle, ticket, C.byref(a), C.byref(b)))
        return a.value, b.value

    def poll(self, ticket: int):
        done = C.c_int()
        led = rt_ledger()
        lat = C.c_double()
        _check(lib().rt_server_poll(self.handle, ticket, C.byref(done), C.byref(led), C.byref(lat)),
               allow_step_limit=True)
        return bool(done.value), (led.as_dict() if done.value else None), lat.value

    def wait(self, ticket: int, timeout_s: float = 600.0) -> None:
        _check(lib().rt_server_wait(self.handle, ticket, float(timeout_s)), allow_step_limit=True)

    def fetch(self, ticket: int):
        ab_shape, img_shape = self.shapes.pop(ticket)
        ab = np.zeros(ab_shape)
        img = np.zeros(img_shape) if img_shape else None
        _check(lib().rt_server_fetch(self.handle, ticket, ab.ctypes.data_as(C.c_void_p),
                                     img.ctypes.data_as(C.c_void_p) if img is not None else None))
        return ab, img

    def release(self, ticket: int) -> None:
        """Drop a finished job's results without copying them out."""
        self.shapes.pop(ticket, None)
        _check(lib().rt_server_fetch(self.handle, ticket, None, None))

    def stats(self):
        used = C.c_size_t()
        q = C.c_int()
        r = C.c_int()
        _check(lib().rt_server_stats(self.handle, C.byref(used), C.byref(q), C.byref(r)))
        return dict(used_bytes=used.value, queued=q.value, running=r.value)

    def close(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.rt_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()
