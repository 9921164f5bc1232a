"""FP64 CPU oracle (test infrastructure only).

A plain, slow restatement of the method in C (``rt_oracle.c``), loaded with
ctypes.  Only the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the CUDA library never
does.  Functions and their paper passages:

* ``Tree``            -- nested-grid hierarchy as a pointer octree (Sect. 2.1)
* ``walk``            -- cell-by-cell ray stepping (Sect. 2.3)
* ``trace``           -- Monte Carlo formal solution with continuous
  absorption and Russian roulette (Sect. 2.3), peel-off images (Sect. 2.4)
* ``dust_temperature``/``dust_emission`` -- equilibrium dust (Sects. 3.2, 4)
* ``lambda_iterate``  -- the Lambda iteration of Eq. 2 with the constant-source
  field computed once and stored (Sect. 3.2)
* ``philox4x32``/``philox4x64`` -- Salmon et al. (2011) counter-based RNG
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rt_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

SRC_POINT, SRC_EXTERNAL, SRC_DUST, SRC_BEAM = 0, 1, 2, 3
EST_CONTINUOUS, EST_ANALOG = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (host code only, portable flags)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "rt_oracle.h"))):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _TreeDesc(C.Structure):
    _fields_ = [("root", C.c_int * 3), ("box", C.c_double * 3), ("n_levels", C.c_int),
                ("n_refined", C.POINTER(C.c_int64)), ("refine_flags", C.POINTER(C.c_uint8)),
                ("density", C.POINTER(C.c_double))]


class _Source(C.Structure):
    _fields_ = [("kind", C.c_int), ("pos", C.c_double * 3), ("dir", C.c_double * 3),
                ("bin_energy", C.POINTER(C.c_double)), ("packets", C.POINTER(C.c_int64)),
                ("emission", C.POINTER(C.c_double)), ("package_energy", C.POINTER(C.c_double))]


class _Optics(C.Structure):
    _fields_ = [("n_lambda", C.c_int), ("kappa_ext", C.POINTER(C.c_double)),
                ("albedo", C.POINTER(C.c_double)), ("g_hg", C.POINTER(C.c_double))]


class _Observers(C.Structure):
    _fields_ = [("n_obs", C.c_int), ("dir", C.POINTER(C.c_double)), ("up", C.POINTER(C.c_double)),
                ("nx", C.c_int), ("ny", C.c_int), ("fov", C.c_double * 2)]


class _Params(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("job", C.c_uint32), ("iter", C.c_uint32),
                ("estimator", C.c_int), ("rr_wmin", C.c_double), ("rr_p", C.c_double),
                ("step_limit", C.c_int64), ("peel_tau_max", C.c_double), ("per_lambda", C.c_int),
                ("n_threads", C.c_int), ("packet_offset", C.c_int64), ("peel_block", C.c_int),
                ("peel_tiles", C.c_int), ("per_level", C.c_int), ("confine_level", C.c_int),
                ("self_absorbed", C.c_void_p), ("self_emitted", C.c_void_p), ("self_count", C.c_void_p),
                ("split_factor", C.c_int), ("split_max_level", C.c_int), ("poly_group", C.c_int),
                ("image_sumsq", C.c_void_p)]


LEDGER_FIELDS = ["emitted", "absorbed", "escaped", "rr_gain", "rr_loss", "killed", "peeled",
                 "n_packets", "n_cross", "n_scatter", "n_peel_cross", "n_killed", "n_peel_out", "n_split"]


class _Ledger(C.Structure):
    _fields_ = [(n, C.c_double) for n in LEDGER_FIELDS]


class _Dust(C.Structure):
    _fields_ = [("n_lambda", C.c_int), ("lambda_um", C.POINTER(C.c_double)),
                ("kappa_abs", C.POINTER(C.c_double)), ("dnu", C.POINTER(C.c_double)),
                ("T_min", C.c_double), ("T_max", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        L.orc_tree_build.restype = C.c_void_p
        L.orc_tree_build.argtypes = [C.POINTER(_TreeDesc)]
        L.orc_tree_free.argtypes = [C.c_void_p]
        L.orc_tree_ncells.restype = C.c_int64
        L.orc_tree_ncells.argtypes = [C.c_void_p]
        L.orc_tree_cells.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_philox4x32.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_philox4x64.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_draw_u32.restype = C.c_uint32
        L.orc_draw_u32.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint64]
        L.orc_walk.restype = C.c_int64
        L.orc_walk.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                               C.c_void_p]
        L.orc_trace.restype = C.c_int
        L.orc_trace.argtypes = [C.c_void_p, C.c_int, C.POINTER(_Source), C.POINTER(_Optics),
                                C.POINTER(_Params), C.POINTER(_Observers), C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(_Ledger)]
        L.orc_dust_packages.restype = C.c_int64
        L.orc_dust_packages.argtypes = [C.c_void_p, C.POINTER(_Source), C.c_int, C.c_int, C.POINTER(_Params),
                                        C.c_void_p]
        L.orc_peel_table.restype = C.c_int64
        L.orc_peel_table.argtypes = [C.c_void_p, C.POINTER(_Observers), C.c_int, C.c_int, C.c_void_p]
        L.orc_peel_point.restype = C.c_int
        L.orc_peel_point.argtypes = [C.c_void_p, C.POINTER(_Optics), C.POINTER(_Observers), C.c_int,
                                     C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]
        L.orc_hg_mu.restype = C.c_double
        L.orc_hg_mu.argtypes = [C.c_double, C.c_double]
        L.orc_hg_phase.restype = C.c_double
        L.orc_hg_phase.argtypes = [C.c_double, C.c_double]
        L.orc_scatter_dir.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_void_p]
        L.orc_emission_per_mass.restype = C.c_double
        L.orc_emission_per_mass.argtypes = [C.POINTER(_Dust), C.c_double]
        L.orc_dust_temperature.restype = C.c_int
        L.orc_dust_temperature.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(_Dust), C.c_int, C.c_void_p]
        L.orc_dust_temperature_weighted.restype = C.c_int
        L.orc_dust_temperature_weighted.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(_Dust), C.c_int,
                                                    C.c_void_p]
        L.orc_dust_emission.restype = C.c_int
        L.orc_dust_emission.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(_Dust), C.c_void_p]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _dp(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class Tree:
    """Pointer octree built from a level-ordered tree description."""

    def __init__(self, desc):
        self._keep = [np.ascontiguousarray(desc.n_refined, dtype=np.int64),
                      np.ascontiguousarray(desc.refine_flags, dtype=np.uint8),
                      np.ascontiguousarray(desc.density, dtype=np.float64)]
        d = _TreeDesc()
        d.root = (C.c_int * 3)(*desc.root)
        d.box = (C.c_double * 3)(*desc.box)
        d.n_levels = len(self._keep[0])
        d.n_refined = _dp(self._keep[0], C.c_int64)
        d.refine_flags = _dp(self._keep[1], C.c_uint8)
        d.density = _dp(self._keep[2], C.c_double)
        self.handle = lib().orc_tree_build(C.byref(d))
        if not self.handle:
            raise ValueError("oracle: inconsistent tree description")
        self.desc = desc
        self.n_cells = int(lib().orc_tree_ncells(self.handle))
        self.box = tuple(desc.box)
        self.root = tuple(desc.root)

    def cells(self):
        lev = np.zeros(self.n_cells, np.uint8)
        leaf = np.zeros(self.n_cells, np.uint8)
        lib().orc_tree_cells(self.handle, _p(lev), _p(leaf))
        return lev, leaf.astype(bool)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.orc_tree_free(self.handle)
            self.handle = None


def philox4x32(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32(_p(c), _p(k), _p(out))
    return out


def philox4x64(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, np.uint64)
    lib().orc_philox4x64(_p(c), _p(k), _p(out))
    return out


def draw_u32(seed, job, iter_, stream, pkt, j) -> int:
    return int(lib().orc_draw_u32(seed, job, iter_, stream, pkt, j))


def walk(tree: Tree, origin, direction, max_seg: int = 100000):
    o = np.ascontiguousarray(origin, np.float64)
    d = np.ascontiguousarray(direction, np.float64)
    cells = np.zeros(max_seg, np.int64)
    lens = np.zeros(max_seg, np.float64)
    marg = np.zeros(max_seg, np.float64)
    n = lib().orc_walk(tree.handle, _p(o), _p(d), max_seg, _p(cells), _p(lens), _p(marg))
    if n < 0:
        raise ValueError("origin outside the box")
    return cells[:n].copy(), lens[:n].copy(), marg[:n].copy()


def hg_mu(g, u):
    return lib().orc_hg_mu(g, u)


def hg_phase(g, mu):
    return lib().orc_hg_phase(g, mu)


def scatter_dir(d, mu, phi):
    dd = np.ascontiguousarray(d, np.float64)
    out = np.zeros(3)
    lib().orc_scatter_dir(_p(dd), mu, phi, _p(out))
    return out


class _Keep:
    def __init__(self):
        self.items = []

    def arr(self, a, dtype):
        a = np.ascontiguousarray(a, dtype=dtype)
        self.items.append(a)
        return a


def _optics(op, keep):
    o = _Optics()
    o.n_lambda = int(len(op.kappa_ext))
    o.kappa_ext = _dp(keep.arr(op.kappa_ext, np.float64), C.c_double)
    o.albedo = _dp(keep.arr(op.albedo, np.float64), C.c_double)
    o.g_hg = _dp(keep.arr(op.g_hg, np.float64), C.c_double)
    return o


def _observers(obs, keep):
    if obs is None:
        return None
    o = _Observers()
    o.n_obs = obs.n_obs
    o.dir = _dp(keep.arr(obs.dirs, np.float64), C.c_double)
    o.up = _dp(keep.arr(obs.ups, np.float64), C.c_double)
    o.nx, o.ny = obs.nx, obs.ny
    o.fov = (C.c_double * 2)(*obs.fov)
    return o


def trace(tree: Tree, sources: Sequence, optics, packets, *, seed: int, job: int = 0, iter_: int = 0,
          estimator: int = EST_CONTINUOUS, rr_wmin: float = 0.0, rr_p: float = 0.9,
          step_limit: int = 0, peel_tau_max: float = 0.0, per_lambda: bool = True,
          observers=None, n_threads: int = 1, validation: bool = False, record: bool = False,
          emission: Optional[np.ndarray] = None, packet_offset: int = 0, peel_block: int = 0,
          peel_tiles: int = 0, per_level: bool = False, confine_level: int = -1, self_absorbed=None,
          self_emitted=None, self_count=None, split_factor: int = 1, split_max_level: int = 255,
          poly_group: int = 1):
    """Run the oracle tracer.

    ``sources`` are ``synth.Source``-like objects (kind "point", "external",
    "beam" or "dust"); ``packets`` is an int or an array [n_src][n_lambda]
    (or [n_lambda]) of packet counts per (source, bin).  ``emission`` is the
    [n_lambda][n_cells] emission table of a dust source.
    Returns a dict with absorbed [bins][n_cells], images, ledger, and the
    optional validation arrays / per-packet records.
    """
    keep = _Keep()
    nl = len(optics.kappa_ext)
    ns = len(sources)
    pk = np.asarray(packets, dtype=np.int64)
    if pk.ndim == 0:
        pk = np.full((ns, nl), int(pk), np.int64)
    elif pk.ndim == 1:
        pk = np.tile(pk, (ns, 1))
    if poly_group > 1:  # packages are counted per group, at its first bin
        pk = np.where((np.arange(nl) % poly_group == 0)[None, :], pk, 0)
    kinds = {"point": SRC_POINT, "external": SRC_EXTERNAL, "dust": SRC_DUST, "beam": SRC_BEAM}
    src_arr = (_Source * ns)()
    for i, s in enumerate(sources):
        S = src_arr[i]
        S.kind = kinds[s.kind]
        S.pos = (C.c_double * 3)(*getattr(s, "pos", (0, 0, 0)))
        S.dir = (C.c_double * 3)(*getattr(s, "dir", (0, 0, 1)))
        be = getattr(s, "bin_energy", None)
        S.bin_energy = _dp(keep.arr(be if be is not None else np.zeros(nl), np.float64), C.c_double)
        S.packets = _dp(keep.arr(pk[i], np.int64), C.c_int64)
        if s.kind == "dust":
            em = emission if emission is not None else s.emission
            S.emission = _dp(keep.arr(em, np.float64), C.c_double)
            if getattr(s, "package_energy", None) is not None:
                S.package_energy = _dp(keep.arr(s.package_energy, np.float64), C.c_double)
    o = _optics(optics, keep)
    prm = _Params(seed=seed, job=job, iter=iter_, estimator=estimator, rr_wmin=rr_wmin, rr_p=rr_p,
                  step_limit=step_limit, peel_tau_max=peel_tau_max, per_lambda=int(per_lambda),
                  n_threads=n_threads, packet_offset=packet_offset, peel_block=peel_block,
                  peel_tiles=peel_tiles, per_level=int(per_level), confine_level=confine_level,
                  self_absorbed=None if self_absorbed is None else self_absorbed.ctypes.data,
                  self_emitted=None if self_emitted is None else self_emitted.ctypes.data,
                  self_count=None if self_count is None else self_count.ctypes.data,
                  split_factor=int(split_factor), split_max_level=int(split_max_level), poly_group=int(poly_group))
    ob = _observers(observers, keep)
    bins = tree.desc.n_levels if per_level else (nl if per_lambda else 1)
    nc = tree.n_cells
    absorbed = np.zeros((bins, nc))
    images = None
    if ob is not None:
        images = np.zeros((observers.n_obs, bins, observers.ny, observers.nx))
    sumsq = np.zeros((bins, nc)) if validation else None
    hits = np.zeros((bins, nc)) if validation else None
    image_sumsq = np.zeros_like(images) if (validation and images is not None) else None
    prm.image_sumsq = None if image_sumsq is None else image_sumsq.ctypes.data
    # a dust source sends its packages per cell: their number is known only
    # from the emission (within one per cell of packets * E_bc / E_b)
    traced = pk.copy()
    for i, s in enumerate(sources):
        if s.kind == "dust":
            actual = np.zeros(nl, np.int64)
            if lib().orc_dust_packages(tree.handle, C.byref(src_arr[i]), i, nl, C.byref(prm),
                                       actual.ctypes.data) < 0:
                raise RuntimeError("orc_dust_packages failed")
            traced[i] = actual
    npk = int(traced.sum())
    rec = np.zeros((npk, 10)) if record else None
    led = _Ledger()
    rc = lib().orc_trace(tree.handle, ns, src_arr, C.byref(o), C.byref(prm),
                         C.byref(ob) if ob is not None else None, _p(absorbed),
                         _p(images) if images is not None else None,
                         _p(sumsq) if validation else None, _p(hits) if validation else None,
                         _p(rec) if record else None, C.byref(led))
    if rc != 0:
        raise RuntimeError(f"orc_trace failed: {rc}")
    return dict(absorbed=absorbed, images=images, sumsq=sumsq, hits=hits, rec=rec, image_sumsq=image_sumsq,
                ledger={n: getattr(led, n) for n in LEDGER_FIELDS})


def peel_table(tree: Tree, observers, block: int, tiles: int) -> np.ndarray:
    """Extinction tables of the accelerated peel-off (Sect. 2.4): column
    densities from block-face tile centres to the model border per observer
    (layout in rt_oracle.h)."""
    keep = _Keep()
    ob = _observers(observers, keep)
    n = lib().orc_peel_table(tree.handle, C.byref(ob), int(block), int(tiles), None)
    if n < 0:
        raise ValueError("orc_peel_table: bad arguments")
    out = np.zeros(max(n, 1))
    lib().orc_peel_table(tree.handle, C.byref(ob), int(block), int(tiles), _p(out))
    return out[:n]


def peel_point(tree: Tree, optics, observers, bin_: int, x_cm, d_in, W, per_lambda=True):
    keep = _Keep()
    o = _optics(optics, keep)
    ob = _observers(observers, keep)
    bins = len(optics.kappa_ext) if per_lambda else 1
    images = np.zeros((observers.n_obs, bins, observers.ny, observers.nx))
    x = keep.arr(x_cm, np.float64)
    d = keep.arr(d_in, np.float64)
    lib().orc_peel_point(tree.handle, C.byref(o), C.byref(ob), bin_, int(per_lambda), _p(x), _p(d),
                         float(W), _p(images))
    return images


def _dust(lambda_um, kappa_abs, dnu, T_min, T_max, keep):
    d = _Dust()
    d.n_lambda = len(lambda_um)
    d.lambda_um = _dp(keep.arr(lambda_um, np.float64), C.c_double)
    d.kappa_abs = _dp(keep.arr(kappa_abs, np.float64), C.c_double)
    d.dnu = _dp(keep.arr(dnu, np.float64), C.c_double)
    d.T_min, d.T_max = T_min, T_max
    return d


def emission_per_mass(lambda_um, kappa_abs, dnu, T, T_min=2.7, T_max=3000.0) -> float:
    keep = _Keep()
    d = _dust(lambda_um, kappa_abs, dnu, T_min, T_max, keep)
    return lib().orc_emission_per_mass(C.byref(d), float(T))


def dust_temperature(tree: Tree, absorbed_total, lambda_um, kappa_abs, dnu, T_min=2.7, T_max=3000.0,
                     n_threads=1) -> np.ndarray:
    keep = _Keep()
    d = _dust(lambda_um, kappa_abs, dnu, T_min, T_max, keep)
    A = keep.arr(absorbed_total, np.float64)
    T = np.zeros(tree.n_cells)
    rc = lib().orc_dust_temperature(tree.handle, _p(A), C.byref(d), n_threads, _p(T))
    if rc != 0:
        raise RuntimeError("orc_dust_temperature failed")
    return T


def dust_temperature_weighted(tree: Tree, rhs, weights, lambda_um, kappa_abs, dnu, T_min=2.7, T_max=3000.0,
                              n_threads=1) -> np.ndarray:
    """Per leaf the T with sum_b weights[b][c] E_b(T) = rhs[c] (bisection)."""
    keep = _Keep()
    d = _dust(lambda_um, kappa_abs, dnu, T_min, T_max, keep)
    r = keep.arr(rhs, np.float64)
    w = keep.arr(weights, np.float64)
    T = np.zeros(tree.n_cells)
    rc = lib().orc_dust_temperature_weighted(tree.handle, _p(r), _p(w), C.byref(d), n_threads, _p(T))
    if rc != 0:
        raise RuntimeError("orc_dust_temperature_weighted failed")
    return T


def dust_emission(tree: Tree, T, lambda_um, kappa_abs, dnu) -> np.ndarray:
    keep = _Keep()
    d = _dust(lambda_um, kappa_abs, dnu, 2.7, 3000.0, keep)
    Tt = keep.arr(T, np.float64)
    em = np.zeros((len(lambda_um), tree.n_cells))
    lib().orc_dust_emission(tree.handle, _p(Tt), C.byref(d), _p(em))
    return em


def packets_by_energy(energy: np.ndarray, total: int) -> np.ndarray:
    """Packets per bin proportional to the bin energy (at least one packet in
    every bin that emits), so that packages carry near-equal weights
    (Sect. 4.2)."""
    e = np.asarray(energy, np.float64)
    tot = e.sum()
    n = np.floor(total * e / tot).astype(np.int64) if tot > 0 else np.zeros(e.size, np.int64)
    n[(e > 0) & (n == 0)] = 1
    return n


def dust_packages(tree: Tree, emission, packets, *, seed: int, job: int = 0, iter_: int = 0, src_index: int = 0,
                  package_energy=None) -> np.ndarray:
    """Packages per bin that a dust source with this emission sends (see
    orc_dust_packages): within one per emitting cell of ``packets``."""
    keep = _Keep()
    em = keep.arr(emission, np.float64)
    nl = em.shape[0]
    pk = keep.arr(np.broadcast_to(np.asarray(packets, np.int64), (nl,)), np.int64)
    S = _Source(kind=SRC_DUST)
    S.packets = _dp(pk, C.c_int64)
    S.emission = _dp(em, C.c_double)
    if package_energy is not None:
        S.package_energy = _dp(keep.arr(package_energy, np.float64), C.c_double)
    prm = _Params(seed=seed, job=job, iter=iter_)
    out = np.zeros(nl, np.int64)
    if lib().orc_dust_packages(tree.handle, C.byref(S), src_index, nl, C.byref(prm), out.ctypes.data) < 0:
        raise RuntimeError("orc_dust_packages failed")
    return out


class _DustSource:
    """Dust emission [n_lambda][n_cells]: each cell sends packages in
    proportion to its emission in each bin (see orc_dust_packages);
    ``package_energy`` [n_lambda], if given, fixes the energy of one package
    (else the bin's emission / packages)."""
    kind = "dust"

    def __init__(self, emission, package_energy=None):
        self.emission = emission
        self.package_energy = package_energy
        self.bin_energy = None


def lambda_iterate(tree: Tree, star, optics, packets_star, packets_dust, *, seed: int, T_min=2.7,
                   T_max=3000.0, max_iter=30, tol=1e-3, min_hits=1000.0, n_threads=1, dust_per_bin=False,
                   **trace_kw):
    """Lambda iteration (Eq. 2): the field of the constant sources is computed
    once and stored (Sect. 3.2); each iteration re-emits the dust with the
    current temperatures, traces the dust photons, and solves the new
    temperatures from the sum of both fields.  The dust packets reuse the
    same random streams every iteration (iteration index kept out of the
    key), so that the change in T between iterations measures convergence
    rather than Monte Carlo noise.  Stops when max dT/T over cells with at
    least ``min_hits`` packet hits is below ``tol`` or after ``max_iter``.
    ``dust_per_bin``: ``packets_dust`` packages in every emitting bin instead
    of a total spread in proportion to the bin emission."""
    kabs = (1 - np.asarray(optics.albedo)) * np.asarray(optics.kappa_ext)
    lam = np.asarray(optics.lambda_um)
    dnu = np.asarray(optics.dnu)
    r = trace(tree, [star], optics, packets_star, seed=seed, iter_=0, per_lambda=False,
              n_threads=n_threads, validation=True, **trace_kw)
    A_star = r["absorbed"][0]
    hits = r["hits"][0]
    T = dust_temperature(tree, A_star, lam, kabs, dnu, T_min, T_max, n_threads)
    history = []
    for it in range(1, max_iter + 1):
        em = dust_emission(tree, T, lam, kabs, dnu)
        if dust_per_bin:
            npk = np.where(em.sum(axis=1) > 0, packets_dust, 0).astype(np.int64)
        else:
            npk = packets_by_energy(em.sum(axis=1), packets_dust)
        rd = trace(tree, [_DustSource(em)], optics, npk, seed=seed, iter_=1, per_lambda=False,
                   n_threads=n_threads, validation=True, **trace_kw)
        A = A_star + rd["absorbed"][0]
        Tn = dust_temperature(tree, A, lam, kabs, dnu, T_min, T_max, n_threads)
        mask = (hits + rd["hits"][0]) >= min_hits
        rel = np.abs(Tn - T)[mask] / np.maximum(T[mask], 1e-300)
        dmax = float(rel.max()) if rel.size else 0.0
        history.append(dmax)
        T = Tn
        if dmax < tol:
            break
    return T, history


def lambda_subiterate(tree: Tree, star, optics, packets_star, packets_dust, *, seed: int, schedule,
                      sub_level: int, T_min=2.7, T_max=3000.0, min_hits=1000.0, n_threads=1,
                      dust_per_bin=False, ali=False, ali_min_packages=100, ali_max_lambda=0.999, **trace_kw):
    """Lambda iteration with subiterations (Sect. 3.2, App. B).  The field of
    the constant sources is computed once.  The dust field is kept in one
    array per grid level i (Eq. 9): I_i holds what packages deposited after
    reaching, as their shallowest grid, one of level i.  A step is either
    "full" (dust emitted from every cell, all I_i replaced) or "sub", a
    subiteration of every subtree below a refined cell of level
    ``sub_level`` = L: dust emitted only from cells of level > L, packages
    leave the run where they reach a grid of level <= L, and only I_i for
    i > L are replaced.  After each step T follows from I_stars + sum_i I_i.
    ``ali``: the accelerated Lambda iteration with the diagonal operator of
    Eq. 3, per frequency (Sect. 3.1: the system decouples into one equation
    per cell with N_freq unknowns): each step also sums, per bin and cell,
    the energy the cell's own packages leave in it (self_b) and the energy
    they carried (emitted_b), and per cell their number; Lambda_b =
    self_b / emitted_b is the fraction of the cell's bin-b emission it
    re-absorbs, capped at ``ali_max_lambda``, and T solves
    sum_b (1 - Lambda_b) E_b(T) = A - sum_b Lambda_b emitted_b.  The
    diagonal operator is used in the cells that sent at least
    ``ali_min_packages`` packages; the others take the plain step, whose
    expectation includes their rare self-absorbed packages.  A bin in which
    such a cell sent no package has no estimate of its own; since a cell
    re-absorbs more of its emission the more opaque it is, the bin takes
    the largest Lambda_j of the cell's sampled bins j with kappa_abs,j <=
    kappa_abs,b (0 if there is none) rather than 0, which would count that
    bin's emission at T as escaping in full.
    Returns T and the per-step max dT/T over cells with >= ``min_hits`` hits."""
    kabs = (1 - np.asarray(optics.albedo)) * np.asarray(optics.kappa_ext)
    lam = np.asarray(optics.lambda_um)
    dnu = np.asarray(optics.dnu)
    r = trace(tree, [star], optics, packets_star, seed=seed, iter_=0, per_lambda=False,
              n_threads=n_threads, validation=True, **trace_kw)
    A_star = r["absorbed"][0]
    hits = r["hits"][0]
    T = dust_temperature(tree, A_star, lam, kabs, dnu, T_min, T_max, n_threads)
    level, _ = tree.cells()
    L = int(sub_level)
    I = np.zeros((tree.desc.n_levels, tree.n_cells))
    history = []
    for step in schedule:
        em = dust_emission(tree, T, lam, kabs, dnu)
        e_bin = em.sum(axis=1)
        if dust_per_bin:
            npk = np.where(e_bin > 0, packets_dust, 0).astype(np.int64)
        else:
            npk = packets_by_energy(e_bin, packets_dust)
        # the package energy of a full step; a subiteration sends from its
        # cells the packages a full step would (App. B), with the same streams
        w = np.where(npk > 0, e_bin / np.maximum(npk, 1), 0.0)
        if step == "sub":
            em = em * (level > L)[None, :]
        elif step != "full":
            raise ValueError("schedule entries are 'full' or 'sub'")
        nlam = len(optics.kappa_ext)
        self_abs = np.zeros((nlam, tree.n_cells)) if ali else None
        self_emit = np.zeros((nlam, tree.n_cells)) if ali else None
        self_n = np.zeros(tree.n_cells) if ali else None
        rd = trace(tree, [_DustSource(em, package_energy=w)], optics, npk, seed=seed, iter_=1, per_lambda=False,
                   n_threads=n_threads, validation=True, per_level=True,
                   confine_level=L if step == "sub" else -1, self_absorbed=self_abs, self_emitted=self_emit,
                   self_count=self_n,
                   **trace_kw)
        if step == "full":
            I[:] = rd["absorbed"]
        else:
            I[L + 1:] = rd["absorbed"][L + 1:]
        A = A_star + I.sum(axis=0)
        if ali:
            on = self_n >= max(ali_min_packages, 1)
            use = on[None, :] & (self_emit > 0)
            lam_s = np.minimum(np.where(use, self_abs / np.where(use, self_emit, 1.0), 0.0), ali_max_lambda)
            lam_b = lam_s.copy()
            for b in range(nlam):
                below = kabs <= kabs[b]
                env = np.where(use[below], lam_s[below], 0.0).max(axis=0)
                lam_b[b] = np.where(on & ~use[b], env, lam_s[b])
            rhs = A - (lam_b * self_emit).sum(axis=0)
            Tn = dust_temperature_weighted(tree, rhs, 1.0 - lam_b, lam, kabs, dnu, T_min, T_max, n_threads)
        else:
            Tn = dust_temperature(tree, A, lam, kabs, dnu, T_min, T_max, n_threads)
        mask = (hits + rd["hits"].sum(axis=0)) >= min_hits
        rel = np.abs(Tn - T)[mask] / np.maximum(T[mask], 1e-300)
        history.append(float(rel.max()) if rel.size else 0.0)
        T = Tn
    return T, history, I
