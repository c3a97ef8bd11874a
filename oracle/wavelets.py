"""SARA dictionary Psi^dagger = [db1, ..., db8, Dirac] / sqrt(9) (Section 2.3.1), float64.

Conventions (the paper gives the dictionary and the faceting halo range only):
  * Daubechies filter of order N (length F = 2N), extremal phase: built by
    spectral factorisation of |H|^2 = 2 cos^{2N}(w/2) P_N(sin^2(w/2)),
    P_N(y) = sum_{k<N} C(N-1+k, k) y^k, keeping for each root y_i of P_N the root
    z_i of z + 1/z = 2 - 4 y_i with |z_i| < 1, so that
    H(w) = c (1 + w)^N prod_i (1 - z_i w), w = z^{-1}, sum h = sqrt(2);
    high-pass g[k] = (-1)^k h[F-1-k].
  * one analysis level, 1-D: zero-padded full convolution sampled at odd
    indices, c[k] = sum_t f[t] a[2k+1-t], k = 0..floor((m+F-1)/2)-1;
    synthesis is its exact transpose, a[i] = sum_k f[2k+1-i] c[k].
  * 2-D level: filter along columns (x, last axis) then rows (y); subbands in
    storage order d0 = (y: h, x: g), d1 = (y: g, x: h), d2 = (y: g, x: g),
    the approximation LL = (y: h, x: h) feeds the next level.
  * 4 levels; coefficient vector of one basis, per channel:
    [lvl1 d0, d1, d2][lvl2 d0, d1, d2][lvl3 ...][lvl4 d0, d1, d2][LL4], each
    subband row-major; the dictionary concatenates db1..db8 then Dirac (the
    image itself); everything is divided by 3 = sqrt(9).
"""
from __future__ import annotations

import math

import numpy as np

LEVELS = 4
NBASES = 9  # db1..db8 + Dirac


def daubechies(N: int) -> np.ndarray:
    """Extremal-phase Daubechies scaling filter h of order N (length 2N)."""
    if N == 1:
        return np.array([1.0, 1.0]) / math.sqrt(2.0)
    # P_N(y) coefficients, highest degree first for numpy.roots
    p = [math.comb(N - 1 + k, k) for k in range(N)]
    yr = np.roots(p[::-1])
    poly = np.array([1.0 + 0j])
    for y in yr:
        b = 2.0 - 4.0 * y
        disc = np.sqrt(b * b - 4.0 + 0j)
        z1, z2 = (b + disc) / 2.0, (b - disc) / 2.0
        z = z1 if abs(z1) < 1.0 else z2
        poly = np.convolve(poly, np.array([1.0, -z]))      # (1 - z w)
    for _ in range(N):
        poly = np.convolve(poly, np.array([1.0, 1.0]))     # (1 + w)
    h = poly.real
    return h * (math.sqrt(2.0) / h.sum())


def highpass(h: np.ndarray) -> np.ndarray:
    F = h.size
    return np.array([(-1) ** k * h[F - 1 - k] for k in range(F)])


def analysis_1d(a: np.ndarray, f: np.ndarray, axis: int) -> np.ndarray:
    """c[k] = sum_t f[t] a[2k+1-t] along `axis` (zero outside the signal)."""
    a = np.moveaxis(a, axis, -1)
    m, F = a.shape[-1], f.size
    full = np.zeros(a.shape[:-1] + (m + F - 1,), dtype=a.dtype)
    for t in range(F):
        full[..., t:t + m] += f[t] * a
    c = full[..., 1::2]
    assert c.shape[-1] == (m + F - 1) // 2
    return np.moveaxis(c, -1, axis)


def synthesis_1d(c: np.ndarray, f: np.ndarray, m: int, axis: int) -> np.ndarray:
    """Transpose of analysis_1d: a[i] = sum_k f[2k+1-i] c[k], i < m."""
    c = np.moveaxis(c, axis, -1)
    F = f.size
    up = np.zeros(c.shape[:-1] + (m + F - 1,), dtype=c.dtype)
    up[..., 1::2] = c
    a = np.zeros(c.shape[:-1] + (m,), dtype=c.dtype)
    for t in range(F):
        a += f[t] * up[..., t:t + m]
    return np.moveaxis(a, -1, axis)


def level_sizes(n1: int, n2: int, F: int, levels: int = LEVELS):
    """[(r_j, c_j)] for j = 0..levels: r_j = floor((r_{j-1} + F - 1) / 2)."""
    sizes = [(n1, n2)]
    for _ in range(levels):
        r, c = sizes[-1]
        sizes.append(((r + F - 1) // 2, (c + F - 1) // 2))
    return sizes


def dwt2(x: np.ndarray, h: np.ndarray, levels: int = LEVELS):
    """Multilevel 2-D analysis of x[..., n1, n2]; returns ([(d0, d1, d2) per level], LL)."""
    g = highpass(h)
    details = []
    a = x
    for _ in range(levels):
        lx = analysis_1d(a, h, -1)
        hx = analysis_1d(a, g, -1)
        ll = analysis_1d(lx, h, -2)
        d0 = analysis_1d(hx, h, -2)
        d1 = analysis_1d(lx, g, -2)
        d2 = analysis_1d(hx, g, -2)
        details.append((d0, d1, d2))
        a = ll
    return details, a


def idwt2(details, ll, h: np.ndarray, n1: int, n2: int) -> np.ndarray:
    """Exact transpose of dwt2."""
    g = highpass(h)
    sizes = level_sizes(n1, n2, h.size, len(details))
    a = ll
    for j in range(len(details), 0, -1):
        m1, m2 = sizes[j - 1]
        d0, d1, d2 = details[j - 1]
        lx = synthesis_1d(a, h, m1, -2) + synthesis_1d(d1, g, m1, -2)
        hx = synthesis_1d(d0, h, m1, -2) + synthesis_1d(d2, g, m1, -2)
        a = synthesis_1d(lx, h, m2, -1) + synthesis_1d(hx, g, m2, -1)
    return a


def basis_filters():
    return [daubechies(N) for N in range(1, 9)]


def basis_size(n1: int, n2: int, F: int, levels: int = LEVELS) -> int:
    s = level_sizes(n1, n2, F, levels)
    return sum(3 * r * c for (r, c) in s[1:]) + s[-1][0] * s[-1][1]


def n_coefficients(n1: int, n2: int) -> int:
    """I: total SARA coefficients per channel."""
    return sum(basis_size(n1, n2, 2 * N) for N in range(1, 9)) + n1 * n2


def sara_analysis(x: np.ndarray) -> np.ndarray:
    """Psi^dagger x for x[..., n1, n2] -> [..., I] (layout in the module docstring)."""
    n1, n2 = x.shape[-2:]
    lead = x.shape[:-2]
    parts = []
    for h in basis_filters():
        details, ll = dwt2(x, h)
        for (d0, d1, d2) in details:
            for d in (d0, d1, d2):
                parts.append(d.reshape(lead + (-1,)))
        parts.append(ll.reshape(lead + (-1,)))
    parts.append(x.reshape(lead + (-1,)))
    return np.concatenate(parts, axis=-1) / 3.0


def sara_synthesis(w: np.ndarray, n1: int, n2: int) -> np.ndarray:
    """Psi w for w[..., I] -> [..., n1, n2] (exact transpose of sara_analysis)."""
    lead = w.shape[:-1]
    out = np.zeros(lead + (n1, n2))
    off = 0
    for h in basis_filters():
        sizes = level_sizes(n1, n2, h.size)
        details = []
        for j in range(1, LEVELS + 1):
            r, c = sizes[j]
            trio = []
            for _ in range(3):
                trio.append(w[..., off:off + r * c].reshape(lead + (r, c)))
                off += r * c
            details.append(tuple(trio))
        r, c = sizes[-1]
        ll = w[..., off:off + r * c].reshape(lead + (r, c))
        off += r * c
        out += idwt2(details, ll, h, n1, n2)
    out += w[..., off:off + n1 * n2].reshape(lead + (n1, n2))
    off += n1 * n2
    assert off == w.shape[-1]
    return out / 3.0


def coefficient_map(n1: int, n2: int):
    """For each basis b (0..8), level j (1..4) and subband s (0..2, 3 = LL4), the
    (offset, rows, cols) of its block in the coefficient vector."""
    table = {}
    off = 0
    for b in range(8):
        F = 2 * (b + 1)
        sizes = level_sizes(n1, n2, F)
        for j in range(1, LEVELS + 1):
            r, c = sizes[j]
            for s in range(3):
                table[(b, j, s)] = (off, r, c)
                off += r * c
        r, c = sizes[-1]
        table[(b, LEVELS, 3)] = (off, r, c)
        off += r * c
    table[(8, 0, 0)] = (off, n1, n2)
    off += n1 * n2
    return table, off
