"""Spatial faceting of Faceted HyperSARA (Section 2.4.2, Fig. 2), float64.

Tiling: tile i of Q along an axis of length n covers [floor(i n / Q), floor((i+1) n / Q)).
Facet q = (qy, qx), q = qy * Qx + qx.  Facets extend their tile towards the top and
left neighbours only; edge facets without such a neighbour do not extend.

SARA facets (the Prusa exact faceted wavelet transform cited in Section 2.4.2):
  * coefficient ownership per axis and level: tile [a_0, b_0) owns, at level j,
    coefficients [a_j, b_j) with a_j = ceil((a_{j-1} - 1) / 2) (0 for the first
    tile) and b_j likewise from the next tile's start (the last tile runs to the
    end of the level); i.e. coefficient k belongs to the tile holding its newest
    input sample 2k + 1;
  * facet input S_q x: pixels [s_0, b_0) with s_0 = max(0, a_0 - halo); the halo
    is the minimal one computed backwards through the levels,
    s_J = a_J, s_{j-1} = 2 s_j + 2 - F (max over the 8 Daubechies filters);
  * Psi_q^dagger S_q x = owned coefficients of the transform of the image
    restricted to the facet input (pixels outside set to zero);
  * S_q^dagger Psi_q w_q = synthesis of the owned coefficients only, restricted to
    the facet input region.

Nuclear facets: tile extended by o = floor(rho * tile side) pixels to the top and
left (none for the first row/column).  D_q is the outer product of 1-D windows:
on an overlap of width o, pixel i = 0..o-1 counted from the later facet's outer
edge has weight w(i) in the later facet and 1 - w(i) in the earlier one, with
triangular w(i) = (i+1)/(o+1) (Fig. 2 piecewise-linear window) or sine
w(i) = sin^2(pi (i+1) / (2 (o+1))); all other pixels weigh 1, so the weights of
every pixel sum to one.
"""
from __future__ import annotations

import math

import numpy as np

from . import wavelets as wv


def tile_bounds(n: int, Q: int) -> list[int]:
    return [(i * n) // Q for i in range(Q + 1)]


# ---------------------------------------------------------------- SARA facets
def _ceil_half_minus(a: int) -> int:
    """ceil((a - 1) / 2) for integer a >= 0."""
    return -((1 - a) // 2)


def owned_ranges_1d(n: int, Q: int, F: int, levels: int = wv.LEVELS):
    """[[(a_j, b_j) for j = 0..levels] for each tile] along one axis."""
    sizes = [n]
    for _ in range(levels):
        sizes.append((sizes[-1] + F - 1) // 2)
    tb = tile_bounds(n, Q)
    out = []
    for i in range(Q):
        a, b = tb[i], tb[i + 1]
        rng = [(a, b)]
        for j in range(1, levels + 1):
            a = 0 if i == 0 else _ceil_half_minus(a)
            b = sizes[j] if i == Q - 1 else _ceil_half_minus(b)
            rng.append((a, b))
        out.append(rng)
    return out


def sara_halo_start(a_J: int, F: int, levels: int = wv.LEVELS) -> int:
    """Unclipped first pixel needed by a facet whose level-`levels` range starts at a_J."""
    s = a_J
    for _ in range(levels):
        s = 2 * s + 2 - F
    return s


def sara_facet_input_1d(n: int, Q: int, levels: int = wv.LEVELS):
    """[(s_0, b_0)] per tile: facet input interval, max halo over db1..db8."""
    out = []
    for i in range(Q):
        starts = []
        for N in range(1, 9):
            F = 2 * N
            rng = owned_ranges_1d(n, Q, F, levels)[i]
            starts.append(sara_halo_start(rng[levels][0], F, levels))
        a0, b0 = tile_bounds(n, Q)[i], tile_bounds(n, Q)[i + 1]
        s0 = min(starts) if i > 0 else 0
        out.append((max(0, s0), b0))
    return out


def sara_facet_mask(n1, n2, Qy, Qx, qy, qx) -> np.ndarray:
    ry = sara_facet_input_1d(n1, Qy)[qy]
    rx = sara_facet_input_1d(n2, Qx)[qx]
    m = np.zeros((n1, n2), dtype=bool)
    m[ry[0]:ry[1], rx[0]:rx[1]] = True
    return m


def sara_owned_index(n1, n2, Qy, Qx, qy, qx) -> np.ndarray:
    """Indices (into the per-channel coefficient vector) owned by facet (qy, qx)."""
    table, total = wv.coefficient_map(n1, n2)
    idx = []
    for b in range(8):
        F = 2 * (b + 1)
        ry = owned_ranges_1d(n1, Qy, F)[qy]
        rx = owned_ranges_1d(n2, Qx, F)[qx]
        for j in range(1, wv.LEVELS + 1):
            subs = [0, 1, 2] + ([3] if j == wv.LEVELS else [])
            for s in subs:
                off, r, c = table[(b, j, s)]
                (a1, b1), (a2, b2) = ry[j], rx[j]
                rr, cc = np.meshgrid(np.arange(a1, b1), np.arange(a2, b2), indexing="ij")
                idx.append((off + rr * c + cc).ravel())
    off, r, c = table[(8, 0, 0)]
    tb1, tb2 = tile_bounds(n1, Qy), tile_bounds(n2, Qx)
    rr, cc = np.meshgrid(np.arange(tb1[qy], tb1[qy + 1]), np.arange(tb2[qx], tb2[qx + 1]), indexing="ij")
    idx.append((off + rr * c + cc).ravel())
    return np.concatenate(idx)


def sara_facet_analysis(x: np.ndarray, Qy: int, Qx: int, qy: int, qx: int):
    """Psi_q^dagger S_q x: (owned indices, coefficients [..., |owned|])."""
    n1, n2 = x.shape[-2:]
    m = sara_facet_mask(n1, n2, Qy, Qx, qy, qx)
    idx = sara_owned_index(n1, n2, Qy, Qx, qy, qx)
    return idx, wv.sara_analysis(x * m)[..., idx]


def sara_facet_synthesis(wq: np.ndarray, idx: np.ndarray, n1, n2, Qy, Qx, qy, qx) -> np.ndarray:
    """S_q^dagger Psi_q w_q: synthesis of the owned coefficients, restricted to the facet input."""
    full = np.zeros(wq.shape[:-1] + (wv.n_coefficients(n1, n2),))
    full[..., idx] = wq
    m = sara_facet_mask(n1, n2, Qy, Qx, qy, qx)
    return wv.sara_synthesis(full, n1, n2) * m


# ------------------------------------------------------------- nuclear facets
def window_weight(i: np.ndarray, o: int, kind: str) -> np.ndarray:
    i = np.asarray(i, dtype=np.float64)
    if kind == "triangular":
        return (i + 1.0) / (o + 1.0)
    if kind == "sine":
        return np.sin(np.pi * (i + 1.0) / (2.0 * (o + 1.0))) ** 2
    raise ValueError(kind)


def nuclear_facets_1d(n: int, Q: int, rho: float, kind: str):
    """[(start, end, window[end-start])] per tile along one axis."""
    tb = tile_bounds(n, Q)
    ov = [0 if i == 0 else int(math.floor(rho * (tb[i + 1] - tb[i]))) for i in range(Q)]
    out = []
    for i in range(Q):
        a, b = tb[i], tb[i + 1]
        start = a - ov[i]
        w = np.ones(b - start)
        if ov[i] > 0:
            w[:ov[i]] = window_weight(np.arange(ov[i]), ov[i], kind)
        if i + 1 < Q and ov[i + 1] > 0:
            o2 = ov[i + 1]
            w[b - o2 - start:] = 1.0 - window_weight(np.arange(o2), o2, kind)
        out.append((start, b, w))
    return out


def nuclear_facets(n1, n2, Qy, Qx, rho, kind):
    """List over q = qy*Qx + qx of dicts with rows (r0, r1), cols (c0, c1) and the 2-D window D_q."""
    fy = nuclear_facets_1d(n1, Qy, rho, kind)
    fx = nuclear_facets_1d(n2, Qx, rho, kind)
    out = []
    for qy in range(Qy):
        for qx in range(Qx):
            r0, r1, wy = fy[qy]
            c0, c1, wx = fx[qx]
            out.append({"rows": (r0, r1), "cols": (c0, c1), "D": np.outer(wy, wx)})
    return out


def sara_facet_analysis_local(x: np.ndarray, Qy: int, Qx: int, qy: int, qx: int):
    """Psi_q^dagger S_q x computed from the facet input region alone (Section 2.4.2).

    Same result and index order as ``sara_facet_analysis``, for images too large to
    transform whole: S_q x is zero outside its input rectangle [s0, b0), so the
    transform of the crop starting at a0 = s0 rounded down to a multiple of 2^LEVELS
    (pixels of the crop before s0 set to zero) holds every owned coefficient; level-j
    index k of the crop is global index k + a0 / 2^j, since the odd-phase decimation
    c[k] = sum_t f[t] a[2k + 1 - t] commutes with shifts by even amounts at every level.
    """
    n1, n2 = x.shape[-2:]
    step = 2 ** wv.LEVELS
    (sy, by), (sx, bx) = sara_facet_input_1d(n1, Qy)[qy], sara_facet_input_1d(n2, Qx)[qx]
    ay, ax = (sy // step) * step, (sx // step) * step
    crop = np.array(x[..., ay:by, ax:bx], dtype=np.float64, copy=True)
    crop[..., : sy - ay, :] = 0.0
    crop[..., :, : sx - ax] = 0.0
    cc = wv.sara_analysis(crop)
    ctab, _ = wv.coefficient_map(by - ay, bx - ax)
    gtab, _ = wv.coefficient_map(n1, n2)
    parts, idx = [], []
    for b in range(8):
        F = 2 * (b + 1)
        ry = owned_ranges_1d(n1, Qy, F)[qy]
        rx = owned_ranges_1d(n2, Qx, F)[qx]
        for j in range(1, wv.LEVELS + 1):
            subs = [0, 1, 2] + ([3] if j == wv.LEVELS else [])
            for s in subs:
                goff, gr, gc = gtab[(b, j, s)]
                coff, cr, ccol = ctab[(b, j, s)]
                (a1, b1), (a2, b2) = ry[j], rx[j]
                oy, ox = ay // 2 ** j, ax // 2 ** j
                assert a1 >= oy and a2 >= ox and b1 - oy <= cr and b2 - ox <= ccol
                rr, cl = np.meshgrid(np.arange(a1, b1), np.arange(a2, b2), indexing="ij")
                idx.append((goff + rr * gc + cl).ravel())
                parts.append(cc[..., coff + (rr - oy) * ccol + (cl - ox)].reshape(x.shape[:-2] + (-1,)))
    tb1, tb2 = tile_bounds(n1, Qy), tile_bounds(n2, Qx)
    goff, gr, gc = gtab[(8, 0, 0)]
    rr, cl = np.meshgrid(np.arange(tb1[qy], tb1[qy + 1]), np.arange(tb2[qx], tb2[qx + 1]), indexing="ij")
    idx.append((goff + rr * gc + cl).ravel())
    parts.append((x[..., rr, cl] / 3.0).reshape(x.shape[:-2] + (-1,)))
    return np.concatenate(idx), np.concatenate(parts, axis=-1)
