"""DDE-extended de-gridding (Section 2.1, the paragraph after Eq. 1), in float64.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU baseline
use this module; the GPU library never does.

Direction-dependent effects (DDEs) multiply the sky seen by visibility m by a pattern
a_m(p).  When that pattern has a compact Fourier-domain representation on the lattice
of the oversampled grid,

    a_m(p) = sum_j K_m[j] exp(-2 pi i (j_r p_r / K1 + j_c p_c / K2)),   j in [-R, R]^2,

(S_d = 2R + 1 coefficients per axis), the visibility of the modulated sky is
y_m = sum_j K_m[j] (F Z x)(t_m + j): the row of G_l is the convolution of the
Kaiser-Bessel kernel with K_m,

    g_m[k] = sum_j K_m[j] phi(t_r - (k_r - j_r)) phi(t_c - (k_c - j_c)),

a (7 + 2R) x (7 + 2R) footprint starting at cell (k0_r - R, k0_c - R), with k0 the first
Kaiser-Bessel tap of t_m (same tap rule as oracle.nufft).  For R = 4 (a 5 x 5 kernel per
antenna, the product of two antennas' patterns giving 9 x 9) the footprint is 15 x 15,
the size the paper quotes.  The adjoint scatters conj(g_m) v_m.

Layout: kern [n_kern][S_d][S_d] complex, first index along grid rows (the v axis), second
along columns (u); kidx [M] selects the kernel of each visibility.
"""
from __future__ import annotations

import numpy as np

from . import nufft as nu


def extended_rows(uv: np.ndarray, kern: np.ndarray, kidx: np.ndarray, K1: int, K2: int):
    """First footprint cell (row, column) of every visibility and its extended row g_m,
    [M][7 + 2R][7 + 2R] complex, from the definition: each DDE coefficient K_m[j] adds a
    Kaiser-Bessel footprint shifted by j."""
    uv = np.asarray(uv, dtype=np.float64)
    kern = np.asarray(kern, dtype=np.complex128)
    S_d = kern.shape[1]
    R = (S_d - 1) // 2
    kr, wr = nu.taps(uv[:, 1] * K1 / (2.0 * np.pi))      # [M][7]
    kc, wc = nu.taps(uv[:, 0] * K2 / (2.0 * np.pi))
    Km = kern[np.asarray(kidx)]                          # [M][S_d][S_d]
    F = nu.J + 2 * R
    g = np.zeros((len(uv), F, F), dtype=np.complex128)
    kb = wr[:, :, None] * wc[:, None, :]                 # [M][7][7]
    for j1 in range(S_d):
        for j2 in range(S_d):
            # cell k = k0 + a + (j - R): footprint coordinate a + j1 (origin k0 - R)
            g[:, j1:j1 + nu.J, j2:j2 + nu.J] += Km[:, j1, j2][:, None, None] * kb
    return kr[:, 0] - R, kc[:, 0] - R, g


def _cells(r0, c0, F, K1, K2):
    rows = (r0[:, None] + np.arange(F)[None, :]) % K1
    cols = (c0[:, None] + np.arange(F)[None, :]) % K2
    return rows[:, :, None], cols[:, None, :]


def degrid(grid: np.ndarray, uv, kern, kidx) -> np.ndarray:
    """u_m = sum_k g_m[k] grid[k mod K]."""
    K1, K2 = grid.shape
    r0, c0, g = extended_rows(uv, kern, kidx, K1, K2)
    rows, cols = _cells(r0, c0, g.shape[1], K1, K2)
    return np.einsum("mij,mij->m", g, grid[rows, cols])


def grid_adjoint(v, uv, kern, kidx, K1: int, K2: int) -> np.ndarray:
    """G^dagger v: scatter-add of conj(g_m[k]) v_m onto the K1 x K2 grid."""
    r0, c0, g = extended_rows(uv, kern, kidx, K1, K2)
    rows, cols = _cells(r0, c0, g.shape[1], K1, K2)
    out = np.zeros((K1, K2), dtype=np.complex128)
    np.add.at(out, (rows, cols), np.conj(g) * np.asarray(v, dtype=np.complex128)[:, None, None])
    return out


def measure(x: np.ndarray, uv, kern, kidx) -> np.ndarray:
    """Phi x = G F Z x with the DDE-extended G, one channel."""
    return degrid(nu.zpad_fft(x), uv, kern, kidx)


def adjoint(v, uv, kern, kidx, n1: int, n2: int) -> np.ndarray:
    """Phi^dagger v = Z^T F^H G^dagger v (complex image; the method takes its real part)."""
    K1, K2 = 2 * n1, 2 * n2
    g = grid_adjoint(v, uv, kern, kidx, K1, K2)
    full = np.fft.ifft2(g) * (K1 * K2)
    rows = nu.pixel_coords(n1) % K1
    cols = nu.pixel_coords(n2) % K2
    s = np.outer(nu.scaling(n1, K1), nu.scaling(n2, K2))
    return s * full[np.ix_(rows, cols)]


def measure_cube(x: np.ndarray, uv, M_l, kern, kidx) -> np.ndarray:
    """Channel by channel; uv, kidx and the result are channel-major."""
    out, off = [], 0
    for l, m in enumerate(M_l):
        out.append(measure(x[l], uv[off:off + m], kern, kidx[off:off + m]))
        off += m
    return np.concatenate(out)


def adjoint_cube_real(v, uv, M_l, kern, kidx, n1: int, n2: int) -> np.ndarray:
    """Re Phi^dagger v channel by channel -> [L][n1][n2]."""
    out, off = [], 0
    for m in M_l:
        out.append(adjoint(v[off:off + m], uv[off:off + m], kern, kidx[off:off + m], n1, n2).real)
        off += m
    return np.stack(out)


def modulated_dft(x: np.ndarray, uv, kern, kidx) -> np.ndarray:
    """The continuous model the extended rows approximate, by brute force: the direct
    DFT (centred pixels, as oracle.nufft.direct_dft) of the sky multiplied by each
    visibility's DDE pattern a_m(p).  Small images only."""
    n1, n2 = x.shape
    K1, K2 = 2 * n1, 2 * n2
    kern = np.asarray(kern, dtype=np.complex128)
    R = (kern.shape[1] - 1) // 2
    pr, pc = nu.pixel_coords(n1), nu.pixel_coords(n2)
    uv = np.asarray(uv, dtype=np.float64)
    js = np.arange(-R, R + 1)
    er_j = np.exp(-2j * np.pi * np.outer(js, pr) / K1)      # [S_d][n1]
    ec_j = np.exp(-2j * np.pi * np.outer(js, pc) / K2)      # [S_d][n2]
    out = np.empty(len(uv), dtype=np.complex128)
    for m in range(len(uv)):
        a = np.einsum("ij,ir,jc->rc", kern[kidx[m]], er_j, ec_j)   # pattern a_m(p)
        e = np.outer(np.exp(-1j * uv[m, 1] * pr), np.exp(-1j * uv[m, 0] * pc))
        out[m] = np.sum(x * a * e)
    return out


__all__ = ["extended_rows", "degrid", "grid_adjoint", "measure", "adjoint", "measure_cube",
           "adjoint_cube_real", "modulated_dft"]
