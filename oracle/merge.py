"""Oracle (test infrastructure): the hierarchical model built bottom-up from
a full-resolution cube (Sect. 4.1).

Only tests/, the package's smoke check and bench.py's CPU baseline use this
module; the library never imports it.

Cells of the full-resolution cube are combined, eight at a time, into the
cell of the next coarser level when (a) all eight are themselves undivided,
(b) the combined cell's optical thickness kappa * rho_mean * h is at most
tau_max (Sect. 4.1: 0.05 in the V band), and (c) the density contrast
rho_max / rho_min over all the full-resolution cells it would contain is
below contrast_max (Sect. 4.1: 30).  The combined density is the mean of the
eight (mass is conserved: equal volumes), summed in octant order
o = ox + 2 oy + 4 oz.  The root cells (level 0) always exist.

The result is a level-ordered tree description: the root cells x-fastest,
then level by level the eight children of each divided cell in the order of
their parents, in octant order.
"""
from __future__ import annotations

import numpy as np


def _children(a, o):
    """The octant-o children of every cell of the next coarser level."""
    ox, oy, oz = o & 1, (o >> 1) & 1, (o >> 2) & 1
    return a[oz::2, oy::2, ox::2]


def merge_uniform(rho, root, box, kappa, tau_max=0.05, contrast_max=30.0):
    """rho: [nz][ny][nx] full-resolution densities (x fastest), n = root * 2^L
    per axis.  Returns (n_refined [L+1], refine_flags, density) in level
    order, plus the per-level arrays (mean, leaf) for the tests."""
    rho = np.asarray(rho, dtype=np.float64)
    root = tuple(int(r) for r in root)
    nz, ny, nx = rho.shape
    L = 0
    while root[0] << L < nx:
        L += 1
    if (root[0] << L, root[1] << L, root[2] << L) != (nx, ny, nz):
        raise ValueError("the cube must have root * 2^L cells per axis")
    h0 = box[0] / root[0]
    mean = [None] * (L + 1)
    mn = [None] * (L + 1)
    mx = [None] * (L + 1)
    leaf = [None] * (L + 1)
    mean[L], mn[L], mx[L] = rho, rho, rho
    leaf[L] = np.ones(rho.shape, dtype=bool)
    for l in range(L - 1, -1, -1):
        s = mean[l + 1]
        acc = _children(s, 0).copy()
        for o in range(1, 8):
            acc = acc + _children(s, o)
        m = acc / 8.0
        lo = _children(mn[l + 1], 0)
        hi = _children(mx[l + 1], 0)
        all_leaf = _children(leaf[l + 1], 0)
        for o in range(1, 8):
            lo = np.minimum(lo, _children(mn[l + 1], o))
            hi = np.maximum(hi, _children(mx[l + 1], o))
            all_leaf = all_leaf & _children(leaf[l + 1], o)
        h = h0 * 0.5 ** l
        tau_ok = kappa * m * h <= tau_max
        contrast_ok = np.where(lo > 0, hi < contrast_max * lo, hi == 0)
        mean[l], mn[l], mx[l] = m, lo, hi
        leaf[l] = all_leaf & tau_ok & contrast_ok
    # level-ordered description
    flags, dens, n_ref = [], [], []
    cur = np.arange(root[0] * root[1] * root[2])          # x-fastest root cells
    cz, cy, cx = cur // (root[0] * root[1]), (cur // root[0]) % root[1], cur % root[0]
    for l in range(L + 1):
        f = ~leaf[l][cz, cy, cx]
        flags.append(f.astype(np.uint8))
        dens.append(mean[l][cz, cy, cx])
        n_ref.append(int(f.sum()))
        if l == L or n_ref[-1] == 0:
            break
        px, py, pz = cx[f], cy[f], cz[f]
        o = np.arange(8)
        cx = (2 * px[:, None] + (o & 1)[None, :]).ravel()
        cy = (2 * py[:, None] + ((o >> 1) & 1)[None, :]).ravel()
        cz = (2 * pz[:, None] + ((o >> 2) & 1)[None, :]).ravel()
    return (np.asarray(n_ref, dtype=np.int64), np.concatenate(flags), np.concatenate(dens)), (mean, leaf)
