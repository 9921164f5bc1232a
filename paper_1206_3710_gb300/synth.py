"""Seeded synthetic model generators (input data only).

This module builds the *inputs* of the radiative-transfer method: hierarchical
(2x2x2-refined) density trees, wavelength grids, dust optical properties,
source spectra and observer geometry.  It holds none of the transport
arithmetic (no ray stepping, no estimator, no temperature solve): both the
CUDA library and the CPU oracle consume what it produces.

Model families (Sect. 4 of Lunttila & Juvela describes the paper's own test
models; these are seeded stand-ins with the shapes and distributions of those
workloads, because the paper's MHD snapshot, ISRF table and dust model are
not available):

* ``tiny_clump``  -- 16^3 root, one refinement level around a Gaussian clump,
  grey opacity, central point source (small case, oracle finishes in seconds).
* ``cloud``       -- 256^3 root, lognormal density from a Gaussian random
  field with P(k) ~ k^-4, three refinement levels, isotropic external field
  at 20 wavelengths (the molecular-cloud test of Sect. 4.1).
* ``disc``        -- flared circumstellar disc with a 64^3 root refined
  towards the star and the midplane up to 10 levels (Sect. 4.2, Eq. 8 form).
* ``batch_models`` -- a seeded list of small models for batched launches.

Tree layout (the input format of ``rt_build_grid``): cells are listed level by
level.  Level 0 is the root grid in x-fastest order, index ix + rx*(iy +
ry*iz).  Level l+1 lists, for every refined level-l cell in order, its eight
children in octant order ox + 2*oy + 4*oz.  ``refine_flags`` has one byte per
cell (1 = refined), ``density`` one float64 per cell (g/cm^3; values of
refined cells are ignored by consumers).  Coordinates run over
[0, box] in cm on each axis; the root grid has cubic cells.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence

import numpy as np

PC_CM = 3.0856775814913673e18
AU_CM = 1.495978707e13
RSUN_CM = 6.957e10
MICRON_CM = 1.0e-4
C_CGS = 2.99792458e10
H_CGS = 6.62607015e-27
K_CGS = 1.380649e-16
SIGMA_SB = 5.670374419e-5
MH_G = 1.6735575e-24


@dataclasses.dataclass
class TreeDesc:
    root: tuple            # (rx, ry, rz)
    box: tuple             # (bx, by, bz) in cm
    n_refined: np.ndarray  # int64 [n_levels]: refined cells per level
    refine_flags: np.ndarray  # uint8 [n_cells], level order
    density: np.ndarray    # float64 [n_cells], level order (g/cm^3)

    @property
    def n_levels(self) -> int:
        return int(len(self.n_refined))

    @property
    def n_cells(self) -> int:
        return int(self.refine_flags.size)

    def level_counts(self) -> np.ndarray:
        counts = [int(np.prod(self.root))]
        for l in range(self.n_levels - 1):
            counts.append(8 * int(self.n_refined[l]))
        return np.asarray(counts, dtype=np.int64)

    def level_offsets(self) -> np.ndarray:
        c = self.level_counts()
        return np.concatenate([[0], np.cumsum(c)]).astype(np.int64)

    def cell_levels(self) -> np.ndarray:
        c = self.level_counts()
        return np.repeat(np.arange(len(c), dtype=np.uint8), c)


@dataclasses.dataclass
class Optics:
    lambda_um: np.ndarray   # [n_lambda]
    kappa_ext: np.ndarray   # cm^2/g
    albedo: np.ndarray
    g_hg: np.ndarray
    dnu: np.ndarray         # Hz, bin widths used by the dust model

    @property
    def n_lambda(self) -> int:
        return int(self.lambda_um.size)


@dataclasses.dataclass
class Source:
    kind: str                 # "point" | "external" | "dust"
    bin_energy: np.ndarray    # energy per wavelength bin (erg/s or code units)
    pos: tuple = (0.0, 0.0, 0.0)  # cm, point sources


@dataclasses.dataclass
class Observers:
    dirs: np.ndarray   # [n_obs, 3] unit vectors towards each observer
    ups: np.ndarray    # [n_obs, 3]
    nx: int
    ny: int
    fov: tuple         # (fov_x, fov_y) cm

    @property
    def n_obs(self) -> int:
        return int(self.dirs.shape[0])


@dataclasses.dataclass
class Model:
    name: str
    tree: TreeDesc
    optics: Optics
    sources: List[Source]
    observers: Optional[Observers]
    packets_per_bin: int
    seed: int


# --------------------------------------------------------------------------
# generic top-down tree growth
# --------------------------------------------------------------------------

_OCT = np.arange(8)
_OX, _OY, _OZ = _OCT & 1, (_OCT >> 1) & 1, (_OCT >> 2) & 1


def grow_tree(root: Sequence[int], box: Sequence[float], max_level: int,
              rho_fn: Callable, refine_fn: Callable,
              max_cells: Optional[int] = None) -> Optional[TreeDesc]:
    """Grow a level-ordered tree top-down.

    ``rho_fn(level, cx, cy, cz)`` returns the density at the centres of the
    cells with integer coordinates (cx, cy, cz) at ``level``;
    ``refine_fn(level, cx, cy, cz, rho)`` returns a boolean refine mask.
    Returns None if ``max_cells`` would be exceeded.
    """
    rx, ry, rz = (int(v) for v in root)
    hx, hy, hz = box[0] / rx, box[1] / ry, box[2] / rz
    if not (math.isclose(hx, hy, rel_tol=1e-12) and math.isclose(hx, hz, rel_tol=1e-12)):
        raise ValueError("root cells must be cubic")
    cz, cy, cx = np.meshgrid(np.arange(rz, dtype=np.int64), np.arange(ry, dtype=np.int64),
                             np.arange(rx, dtype=np.int64), indexing="ij")
    cx, cy, cz = cx.ravel(), cy.ravel(), cz.ravel()
    flags_all, rho_all, n_ref = [], [], []
    total = 0
    for lev in range(max_level + 1):
        rho = np.asarray(rho_fn(lev, cx, cy, cz), dtype=np.float64)
        if lev < max_level:
            flags = np.asarray(refine_fn(lev, cx, cy, cz, rho), dtype=bool)
        else:
            flags = np.zeros(cx.size, dtype=bool)
        total += cx.size
        if max_cells is not None and total + 8 * int(flags.sum()) > max_cells:
            return None
        flags_all.append(flags.astype(np.uint8))
        rho_all.append(rho)
        n_ref.append(int(flags.sum()))
        if n_ref[-1] == 0:
            break
        px, py, pz = cx[flags], cy[flags], cz[flags]
        cx = (2 * px[:, None] + _OX[None, :]).ravel()
        cy = (2 * py[:, None] + _OY[None, :]).ravel()
        cz = (2 * pz[:, None] + _OZ[None, :]).ravel()
    return TreeDesc(root=(rx, ry, rz), box=tuple(float(b) for b in box),
                    n_refined=np.asarray(n_ref, dtype=np.int64),
                    refine_flags=np.concatenate(flags_all),
                    density=np.concatenate(rho_all))


def uniform_tree(root: Sequence[int], box: Sequence[float], rho: float) -> TreeDesc:
    return grow_tree(root, box, 0, lambda l, x, y, z: np.full(x.size, rho),
                     lambda l, x, y, z, r: np.zeros(x.size, bool))


def random_refined_tree(root: Sequence[int], box: Sequence[float], max_level: int,
                        p_refine: float, seed: int,
                        rho_fn: Optional[Callable] = None) -> TreeDesc:
    """Random refinement pattern (each cell refined with probability p)."""
    rng = np.random.default_rng(seed)
    if rho_fn is None:
        rho_fn = lambda l, x, y, z: rng.uniform(0.5, 1.5, size=x.size)
    return grow_tree(root, box, max_level, rho_fn,
                     lambda l, x, y, z, r: rng.random(x.size) < p_refine)


# --------------------------------------------------------------------------
# wavelengths and dust
# --------------------------------------------------------------------------

def log_lambda_grid(n: int, lo_um: float = 0.1, hi_um: float = 1000.0) -> np.ndarray:
    if n == 1:
        return np.array([0.55])
    return np.logspace(math.log10(lo_um), math.log10(hi_um), n)


def bin_dnu(lambda_um: np.ndarray) -> np.ndarray:
    """Frequency width of each wavelength bin; bin edges sit at the geometric
    midpoints, the outer edges half a log step beyond the end points."""
    lam = np.asarray(lambda_um, dtype=np.float64)
    if lam.size == 1:
        edges = np.array([lam[0] / 1.1, lam[0] * 1.1])
    else:
        mid = np.sqrt(lam[:-1] * lam[1:])
        lo = lam[0] / math.sqrt(lam[1] / lam[0])
        hi = lam[-1] * math.sqrt(lam[-1] / lam[-2])
        edges = np.concatenate([[lo], mid, [hi]])
    nu_edges = C_CGS / (edges * MICRON_CM)
    return nu_edges[:-1] - nu_edges[1:]


def albedo_law(lambda_um: np.ndarray) -> np.ndarray:
    lam = np.asarray(lambda_um, dtype=np.float64)
    x = np.clip(np.log10(lam / 0.1) / 2.0, 0.0, None)
    a = 0.6 * (0.01 / 0.6) ** x
    return np.where(lam > 10.0, 0.01, a)


def powerlaw_dust(lambda_um: np.ndarray, kappa_ref: float, lambda_ref_um: float,
                  g: float = 0.5) -> Optics:
    lam = np.asarray(lambda_um, dtype=np.float64)
    kext = kappa_ref * (lam / lambda_ref_um) ** -1.8
    return Optics(lambda_um=lam, kappa_ext=kext, albedo=albedo_law(lam),
                  g_hg=np.full(lam.size, g), dnu=bin_dnu(lam))


def planck_nu(nu: np.ndarray, T: float) -> np.ndarray:
    x = H_CGS * nu / (K_CGS * T)
    return 2.0 * H_CGS * nu ** 3 / C_CGS ** 2 / np.expm1(x)


def blackbody_star_bins(lambda_um: np.ndarray, T: float, R_cm: float) -> np.ndarray:
    """Luminosity per bin of a blackbody star: 4 pi R^2 * pi B_nu * dnu."""
    nu = C_CGS / (np.asarray(lambda_um) * MICRON_CM)
    return 4.0 * math.pi * R_cm ** 2 * math.pi * planck_nu(nu, T) * bin_dnu(lambda_um)


def axis_observers(n_pix: int, fov: float, which: str = "all6") -> Observers:
    dirs = {"+x": (1, 0, 0), "-x": (-1, 0, 0), "+y": (0, 1, 0), "-y": (0, -1, 0),
            "+z": (0, 0, 1), "-z": (0, 0, -1)}
    names = ["+x", "-x", "+y", "-y", "+z", "-z"] if which == "all6" else [which]
    d = np.array([dirs[n] for n in names], dtype=np.float64)
    ups = np.array([(0, 0, 1) if abs(v[1]) > 0.5 else (0, 1, 0) for v in d], dtype=np.float64)
    return Observers(dirs=d, ups=ups, nx=n_pix, ny=n_pix, fov=(fov, fov))


# --------------------------------------------------------------------------
# C1: tiny clump
# --------------------------------------------------------------------------

def tiny_clump(n_root: int = 16, packets: int = 100_000, seed: int = 1001,
               contrast: float = 100.0, rho_bg: float = 1.0e-21) -> Model:
    L = PC_CM
    sig = 0.1 * L
    rho_c = contrast * rho_bg

    def rho_fn(lev, cx, cy, cz):
        h = L / n_root / (1 << lev)
        x = (cx + 0.5) * h - 0.5 * L
        y = (cy + 0.5) * h - 0.5 * L
        z = (cz + 0.5) * h - 0.5 * L
        return rho_bg + rho_c * np.exp(-(x * x + y * y + z * z) / (2 * sig * sig))

    root_mean = [None]

    def refine_fn(lev, cx, cy, cz, rho):
        if root_mean[0] is None:
            root_mean[0] = float(rho.mean())
        return rho > 2.0 * root_mean[0]

    tree = grow_tree((n_root,) * 3, (L,) * 3, 1, rho_fn, refine_fn)
    # grey opacity normalised so that the analytic optical depth from the
    # centre to the +x face equals 1
    col = rho_bg * 0.5 * L + rho_c * sig * math.sqrt(math.pi / 2) * math.erf(0.5 * L / (math.sqrt(2) * sig))
    kappa = 1.0 / col
    optics = Optics(lambda_um=np.array([0.55]), kappa_ext=np.array([kappa]),
                    albedo=np.array([0.5]), g_hg=np.array([0.0]), dnu=bin_dnu(np.array([0.55])))
    src = Source("point", bin_energy=np.array([1.0]), pos=(0.5 * L,) * 3)
    obs = axis_observers(64, L, "+z")
    return Model("tiny_clump", tree, optics, [src], obs, packets, seed)


# --------------------------------------------------------------------------
# C2: lognormal cloud
# --------------------------------------------------------------------------

def gaussian_random_field(n: int, seed: int, slope: float = -4.0) -> np.ndarray:
    """Periodic unit-variance Gaussian random field on n^3, P(k) ~ k^slope.
    Returned array is indexed [iz, iy, ix]."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((n, n, n))
    f = np.fft.rfftn(white)
    del white
    kz = np.fft.fftfreq(n)[:, None, None]
    ky = np.fft.fftfreq(n)[None, :, None]
    kx = np.fft.rfftfreq(n)[None, None, :]
    k2 = kz * kz + ky * ky + kx * kx
    k2[0, 0, 0] = 1.0
    amp = k2 ** (slope / 4.0)
    amp[0, 0, 0] = 0.0
    f *= amp
    g = np.fft.irfftn(f, s=(n, n, n), axes=(0, 1, 2))
    g -= g.mean()
    g /= g.std()
    return g


def _trilinear_periodic(g: np.ndarray, px, py, pz) -> np.ndarray:
    """Trilinear interpolation of a periodic field sampled at cell centres
    (i + 0.5) in root units, at positions (px, py, pz) in root units."""
    n = g.shape[0]
    out = np.empty(px.size, dtype=np.float64)
    chunk = 1 << 22
    for s in range(0, px.size, chunk):
        qx = px[s:s + chunk] - 0.5
        qy = py[s:s + chunk] - 0.5
        qz = pz[s:s + chunk] - 0.5
        ix0 = np.floor(qx).astype(np.int64)
        iy0 = np.floor(qy).astype(np.int64)
        iz0 = np.floor(qz).astype(np.int64)
        wx, wy, wz = qx - ix0, qy - iy0, qz - iz0
        ix0 %= n; iy0 %= n; iz0 %= n
        ix1, iy1, iz1 = (ix0 + 1) % n, (iy0 + 1) % n, (iz0 + 1) % n
        acc = np.zeros(qx.size)
        for zz, wzz in ((iz0, 1 - wz), (iz1, wz)):
            for yy, wyy in ((iy0, 1 - wy), (iy1, wy)):
                for xx, wxx in ((ix0, 1 - wx), (ix1, wx)):
                    acc += wzz * wyy * wxx * g[zz, yy, xx]
        out[s:s + chunk] = acc
    return out


def cloud(n_root: int = 256, levels: int = 3, seed: int = 1002, n_lambda: int = 20,
          packets_per_bin: int = 10_000_000, threshold_scale: float = 1.0,
          sigma_ln: float = 1.5, box_pc: float = 2.0, n_pix: int = 256,
          tau_mean_V: float = 0.4) -> Model:
    L = box_pc * PC_CM
    rho_unit = 70.0 * 2.8 * MH_G           # n(H2) = 70 cm^-3, mean molecular mass 2.8 m_H
    g = gaussian_random_field(n_root, seed)
    mu = -0.5 * sigma_ln * sigma_ln        # mean of exp(sigma g + mu) is 1

    def rho_fn(lev, cx, cy, cz):
        if lev == 0:
            gv = g[cz, cy, cx]
        else:
            s = 1.0 / (1 << lev)
            gv = _trilinear_periodic(g, (cx + 0.5) * s, (cy + 0.5) * s, (cz + 0.5) * s)
        return rho_unit * np.exp(sigma_ln * gv + mu)

    def refine_fn(lev, cx, cy, cz, rho):
        return rho > threshold_scale * 4.0 ** (lev + 1) * rho_unit

    tree = grow_tree((n_root,) * 3, (L,) * 3, levels, rho_fn, refine_fn)
    lam = log_lambda_grid(n_lambda)
    kV = tau_mean_V / (rho_unit * L)       # mean tau_ext at 0.55 um across the box side
    optics = powerlaw_dust(lam, kV, 0.55, g=0.5)
    # isotropic external field with equal energy per ln(lambda) bin, total 1
    src = Source("external", bin_energy=np.full(n_lambda, 1.0 / n_lambda))
    obs = axis_observers(n_pix, L, "all6")
    return Model("cloud", tree, optics, [src], obs, packets_per_bin, seed)


# --------------------------------------------------------------------------
# C3: circumstellar disc
# --------------------------------------------------------------------------

def disc_density_fn(rho0: float, L: float, r_in_au=0.1, r_out_au=300.0,
                    alpha=2.25, h1_au=0.05, beta=1.125):
    def rho_at(x, y, z):
        """x, y, z in cm relative to the box centre."""
        r = np.sqrt(x * x + y * y) / AU_CM
        h = h1_au * np.maximum(r, 1e-30) ** beta * AU_CM
        with np.errstate(divide="ignore", over="ignore", invalid="ignore"):
            rho = rho0 * np.maximum(r, 1e-30) ** (-alpha) * np.exp(-0.5 * (z / h) ** 2)
        return np.where((r >= r_in_au) & (r <= r_out_au), rho, 0.0)
    return rho_at


def disc(n_root: int = 64, max_level: int = 10, n_lambda: int = 30,
         packets: int = 100_000_000, seed: int = 1003, target_cells: float = 1.0e7,
         tau_mid_1um: float = 1.0e5, box_au: float = 600.0, T_star: float = 4000.0,
         R_star_rsun: float = 2.0, tau_cell_thr: Optional[float] = None,
         max_cells: int = 30_000_000) -> Model:
    L = box_au * AU_CM
    lam = log_lambda_grid(n_lambda)
    r_in, r_out, alpha = 0.1, 300.0, 2.25
    integral = (r_in ** (1 - alpha) - r_out ** (1 - alpha)) / (alpha - 1)   # AU^(1-alpha) * AU
    k1 = 1.0                                  # cm^2/g at 1 um (scale absorbed into rho0)
    rho0 = tau_mid_1um / (k1 * integral * AU_CM)
    optics = powerlaw_dust(lam, k1, 1.0, g=0.5)
    rho_at = disc_density_fn(rho0, L, r_in, r_out, alpha)
    h0 = L / n_root
    star_root = np.array([0.5 * n_root] * 3)

    def rho_fn(lev, cx, cy, cz):
        h = h0 / (1 << lev)
        return rho_at((cx + 0.5) * h - 0.5 * L, (cy + 0.5) * h - 0.5 * L, (cz + 0.5) * h - 0.5 * L)

    def make_refine(thr):
        def refine_fn(lev, cx, cy, cz, rho):
            h = h0 / (1 << lev)
            rmax = rho.copy()
            for ox in (0, 1):
                for oy in (0, 1):
                    for oz in (0, 1):
                        rmax = np.maximum(rmax, rho_at((cx + ox) * h - 0.5 * L, (cy + oy) * h - 0.5 * L,
                                                       (cz + oz) * h - 0.5 * L))
            sc = np.floor(star_root * (1 << lev)).astype(np.int64)
            has_star = (cx == sc[0]) & (cy == sc[1]) & (cz == sc[2])
            return (k1 * rmax * h > thr) | has_star
        return refine_fn

    if tau_cell_thr is None:
        # raise the per-cell optical-depth threshold until the cell count is near target
        lo, hi = 0.0, 8.0   # log10 thresholds
        best = None
        for _ in range(14):
            mid = 0.5 * (lo + hi)
            t = grow_tree((n_root,) * 3, (L,) * 3, max_level, rho_fn, make_refine(10 ** mid),
                          max_cells=max_cells)
            if t is None or t.n_cells > target_cells:
                lo = mid
            else:
                hi = mid
                best = (mid, t)
            if best is not None and abs(best[1].n_cells - target_cells) < 0.1 * target_cells:
                break
        tau_cell_thr = 10 ** best[0]
        tree = best[1]
    else:
        tree = grow_tree((n_root,) * 3, (L,) * 3, max_level, rho_fn, make_refine(tau_cell_thr),
                         max_cells=max_cells)
    Lb = blackbody_star_bins(lam, T_star, R_star_rsun * RSUN_CM)
    src = Source("point", bin_energy=Lb, pos=(0.5 * L,) * 3)
    m = Model("disc", tree, optics, [src], None, packets // n_lambda, seed)
    m.tau_cell_thr = tau_cell_thr
    return m


# --------------------------------------------------------------------------
# C4: batch of small models
# --------------------------------------------------------------------------

def batch_models(n_models: int = 64, seed: int = 1004, n_lambda: int = 16,
                 min_packets: float = 1e5, max_packets: float = 1e7,
                 roots=(32, 64, 128), max_levels: int = 4) -> List[Model]:
    rng = np.random.default_rng(seed)
    out = []
    lam = log_lambda_grid(n_lambda)
    for m in range(n_models):
        n_root = int(rng.choice(roots))
        levels = int(rng.integers(0, max_levels + 1))
        total = float(np.exp(rng.uniform(np.log(min_packets), np.log(max_packets))))
        ppb = max(1, int(total / n_lambda))
        if m % 2 == 0:
            L = PC_CM
            sig = 0.1 * L
            rho_bg = 1e-21

            def rho_fn(lev, cx, cy, cz, L=L, n=n_root, sig=sig, rho_bg=rho_bg):
                h = L / n / (1 << lev)
                x = (cx + 0.5) * h - 0.5 * L
                y = (cy + 0.5) * h - 0.5 * L
                z = (cz + 0.5) * h - 0.5 * L
                return rho_bg * (1 + 100 * np.exp(-(x * x + y * y + z * z) / (2 * sig * sig)))

            def refine_fn(lev, cx, cy, cz, rho, rho_bg=rho_bg):
                return rho > 2.0 * 2.57 * rho_bg * 4.0 ** lev

            tree = grow_tree((n_root,) * 3, (L,) * 3, levels, rho_fn, refine_fn)
            col = rho_bg * 0.5 * L + 100 * rho_bg * sig * math.sqrt(math.pi / 2)
            optics = powerlaw_dust(lam, 1.0 / col, 0.55)
            src = Source("point", bin_energy=np.full(n_lambda, 1.0 / n_lambda), pos=(0.5 * L,) * 3)
        else:
            L = 2 * PC_CM
            rho_unit = 70.0 * 2.8 * MH_G
            g = gaussian_random_field(n_root, int(rng.integers(1 << 30)))

            def rho_fn(lev, cx, cy, cz, g=g, rho_unit=rho_unit):
                if lev == 0:
                    gv = g[cz, cy, cx]
                else:
                    s = 1.0 / (1 << lev)
                    gv = _trilinear_periodic(g, (cx + 0.5) * s, (cy + 0.5) * s, (cz + 0.5) * s)
                return rho_unit * np.exp(1.5 * gv - 1.125)

            def refine_fn(lev, cx, cy, cz, rho, rho_unit=rho_unit):
                return rho > 4.0 ** (lev + 1) * rho_unit

            tree = grow_tree((n_root,) * 3, (L,) * 3, levels, rho_fn, refine_fn)
            optics = powerlaw_dust(lam, 0.4 / (rho_unit * L), 0.55)
            src = Source("external", bin_energy=np.full(n_lambda, 1.0 / n_lambda))
        out.append(Model(f"batch{m}", tree, optics, [src], None, ppb, seed * 1000 + m))
    return out
