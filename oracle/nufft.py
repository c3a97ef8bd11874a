"""Measurement operator Phi_l = G_l F Z of Eq. (1) (Section 2.1), in float64.

Conventions (the paper names only "Kaiser-Bessel, S = 7x7, Fessler 2003"):
  * image x[r][c], r < n1 rows, c < n2 columns; centred pixel coordinates
    p_r = r - n1/2, p_c = c - n2/2;
  * a visibility has (u, v) in rad/pixel, u pairs with the column coordinate,
    v with the row coordinate: the continuous model is
    y = sum_{r,c} x[r][c] exp(-i (u p_c + v p_r))   (direct DFT);
  * Z: scale by s_r s_c, s = 1 / phi_hat(2 pi p / K), zero-pad to K1 x K2 = 2n1 x 2n2;
  * F: 2-D DFT with exp(-2 pi i k p / K);
  * G: per visibility, t = omega K / (2 pi); 7 taps per axis at k_j = floor(t - 3.5) + 1 + j,
    j = 0..6, weight phi(t - k_j), grid index k_j mod K;
  * phi(u) = I0(beta sqrt(1 - (2u/J)^2)) / I0(beta), |u| <= J/2, J = 7, beta = 2.34 J
    (Fessler & Sutton 2003 choice for 2x oversampling);
  * adjoint: exact transpose, x = conj(Z)^T F^H G^T v; the method uses its real part
    (projection on real images, Table 2 last row).
"""
from __future__ import annotations

import math

import numpy as np

J = 7
BETA = 2.34 * J


def kb_kernel(u):
    """Kaiser-Bessel interpolation kernel phi(u), zero outside |u| <= J/2."""
    u = np.asarray(u, dtype=np.float64)
    arg = 1.0 - (2.0 * u / J) ** 2
    inside = arg >= 0.0
    out = np.zeros_like(u)
    out[inside] = np.i0(BETA * np.sqrt(arg[inside])) / np.i0(BETA)
    return out


def kb_kernel_ft(theta):
    """Continuous Fourier transform of phi: int phi(u) exp(-i theta u) du.

    Closed form of the Kaiser-Bessel window transform:
    J sinh(z) / z / I0(beta), z = sqrt(beta^2 - (J theta / 2)^2)
    (sin form when the radicand is negative).
    """
    theta = np.asarray(theta, dtype=np.float64)
    rad = BETA ** 2 - (J * theta / 2.0) ** 2
    out = np.empty_like(theta)
    pos = rad > 0
    z = np.sqrt(np.abs(rad))
    with np.errstate(invalid="ignore", divide="ignore"):
        out[pos] = np.sinh(z[pos]) / z[pos]
        neg = ~pos
        out[neg] = np.where(z[neg] > 0, np.sin(z[neg]) / np.where(z[neg] > 0, z[neg], 1.0), 1.0)
    return J * out / np.i0(BETA)


def pixel_coords(n: int) -> np.ndarray:
    """Centred coordinates p = i - n/2 of pixel indices i = 0..n-1."""
    return np.arange(n) - n // 2


def scaling(n: int, K: int) -> np.ndarray:
    """Diagonal of Z along one axis: s = 1 / phi_hat(2 pi p / K)."""
    return 1.0 / kb_kernel_ft(2.0 * np.pi * pixel_coords(n) / K)


def direct_dft(x: np.ndarray, uv: np.ndarray) -> np.ndarray:
    """y_m = sum_{r,c} x[r][c] exp(-i (u_m p_c + v_m p_r)) (exact model behind Eq. 1)."""
    n1, n2 = x.shape
    pr = pixel_coords(n1)
    pc = pixel_coords(n2)
    uv = np.asarray(uv, dtype=np.float64)
    er = np.exp(-1j * np.outer(uv[:, 1], pr))   # [M][n1]
    ec = np.exp(-1j * np.outer(uv[:, 0], pc))   # [M][n2]
    return np.einsum("mr,rc,mc->m", er, x.astype(np.complex128), ec)


def zpad_fft(x: np.ndarray) -> np.ndarray:
    """F Z x: scale by s_r s_c, place pixel p at grid index p mod K, 2-D DFT (numpy.fft)."""
    n1, n2 = x.shape
    K1, K2 = 2 * n1, 2 * n2
    g = np.zeros((K1, K2), dtype=np.complex128)
    s = np.outer(scaling(n1, K1), scaling(n2, K2))
    rows = pixel_coords(n1) % K1
    cols = pixel_coords(n2) % K2
    g[np.ix_(rows, cols)] = s * x
    return np.fft.fft2(g)


def taps(t: np.ndarray):
    """Tap indices k_j = floor(t - 3.5) + 1 + j and weights phi(t - k_j), j = 0..6."""
    k0 = np.floor(t - J / 2.0).astype(np.int64) + 1
    k = k0[:, None] + np.arange(J)[None, :]
    w = kb_kernel(t[:, None] - k)
    return k, w


def degrid(grid: np.ndarray, uv: np.ndarray) -> np.ndarray:
    """G: y_m = sum_{i,j} phi(t_r - k_i) phi(t_c - k_j) grid[k_i mod K1][k_j mod K2]."""
    K1, K2 = grid.shape
    uv = np.asarray(uv, dtype=np.float64)
    tr = uv[:, 1] * K1 / (2.0 * np.pi)
    tc = uv[:, 0] * K2 / (2.0 * np.pi)
    kr, wr = taps(tr)
    kc, wc = taps(tc)
    vals = grid[(kr % K1)[:, :, None], (kc % K2)[:, None, :]]   # [M][7][7]
    return np.einsum("mi,mj,mij->m", wr, wc, vals)


def grid_adjoint(v: np.ndarray, uv: np.ndarray, K1: int, K2: int) -> np.ndarray:
    """G^T: scatter-add of phi(t_r - k_i) phi(t_c - k_j) v_m onto the K1 x K2 grid."""
    uv = np.asarray(uv, dtype=np.float64)
    tr = uv[:, 1] * K1 / (2.0 * np.pi)
    tc = uv[:, 0] * K2 / (2.0 * np.pi)
    kr, wr = taps(tr)
    kc, wc = taps(tc)
    g = np.zeros((K1, K2), dtype=np.complex128)
    contrib = wr[:, :, None] * wc[:, None, :] * np.asarray(v)[:, None, None]
    np.add.at(g, ((kr % K1)[:, :, None], (kc % K2)[:, None, :]), contrib)
    return g


def measure(x: np.ndarray, uv: np.ndarray) -> np.ndarray:
    """Phi x = G F Z x for one channel (Eq. 1)."""
    return degrid(zpad_fft(x), uv)


def adjoint(v: np.ndarray, uv: np.ndarray, n1: int, n2: int) -> np.ndarray:
    """Phi^dagger v = Z^T F^H G^T v (complex image; the method uses its real part)."""
    K1, K2 = 2 * n1, 2 * n2
    g = grid_adjoint(v, uv, K1, K2)
    full = np.fft.ifft2(g) * (K1 * K2)          # sum_k g[k] exp(+2 pi i k p / K)
    rows = pixel_coords(n1) % K1
    cols = pixel_coords(n2) % K2
    s = np.outer(scaling(n1, K1), scaling(n2, K2))
    return s * full[np.ix_(rows, cols)]


def measure_sampled(x: np.ndarray, uv: np.ndarray) -> np.ndarray:
    """Phi x (Eq. 1) at a few visibilities without an FFT: the 7 x 7 grid values each
    visibility reads are DFT sums of the scaled image, taken as E_r (s x) E_c^T with
    E[k][p] = exp(-2 pi i k p / K) over the tap rows and columns, then weighted by the
    Kaiser-Bessel taps.  For checks of large images at sampled outputs."""
    n1, n2 = x.shape
    K1, K2 = 2 * n1, 2 * n2
    uv = np.asarray(uv, dtype=np.float64)
    kr, wr = taps(uv[:, 1] * K1 / (2.0 * np.pi))          # [S][7]
    kc, wc = taps(uv[:, 0] * K2 / (2.0 * np.pi))
    sx = np.outer(scaling(n1, K1), scaling(n2, K2)) * x
    er = np.exp(-2j * np.pi * np.outer(kr.ravel(), pixel_coords(n1)) / K1)   # [7S][n1]
    ec = np.exp(-2j * np.pi * np.outer(kc.ravel(), pixel_coords(n2)) / K2)   # [7S][n2]
    rows = (er @ sx).reshape(len(uv), J, n2)                                  # [S][7][n2]
    g = np.einsum("mic,mjc->mij", rows, ec.reshape(len(uv), J, n2))
    return np.einsum("mi,mj,mij->m", wr, wc, g)


def adjoint_real_sampled(v: np.ndarray, uv: np.ndarray, n1: int, n2: int, pix) -> np.ndarray:
    """Re Phi^dagger v at a few pixels (r, c) by direct summation over visibilities and
    taps: s_r s_c Re sum_m v_m (sum_i w_i e^{2 pi i k_i p_r / K1}) (sum_j w_j e^{2 pi i k_j p_c / K2})."""
    K1, K2 = 2 * n1, 2 * n2
    uv = np.asarray(uv, dtype=np.float64)
    v = np.asarray(v, dtype=np.complex128)
    kr, wr = taps(uv[:, 1] * K1 / (2.0 * np.pi))
    kc, wc = taps(uv[:, 0] * K2 / (2.0 * np.pi))
    sr, sc = scaling(n1, K1), scaling(n2, K2)
    pr, pc = pixel_coords(n1), pixel_coords(n2)
    out = np.empty(len(pix))
    for i, (r, c) in enumerate(pix):
        ar = (wr * np.exp(2j * np.pi * kr * pr[r] / K1)).sum(axis=1)
        ac = (wc * np.exp(2j * np.pi * kc * pc[c] / K2)).sum(axis=1)
        out[i] = sr[r] * sc[c] * np.real(np.sum(v * ar * ac))
    return out


def measure_cube(x: np.ndarray, uv: np.ndarray, M_l) -> np.ndarray:
    """Phi applied channel by channel; uv and the result are channel-major."""
    out, off = [], 0
    for l, m in enumerate(M_l):
        out.append(measure(x[l], uv[off:off + m]))
        off += m
    return np.concatenate(out)


def adjoint_cube_real(v: np.ndarray, uv: np.ndarray, M_l, n1: int, n2: int) -> np.ndarray:
    """Re Phi^dagger v channel by channel -> [L][n1][n2]."""
    out, off = [], 0
    for m in M_l:
        out.append(adjoint(v[off:off + m], uv[off:off + m], n1, n2).real)
        off += m
    return np.stack(out)


__all__ = ["J", "BETA", "kb_kernel", "kb_kernel_ft", "pixel_coords", "scaling", "direct_dft",
           "zpad_fft", "taps", "degrid", "grid_adjoint", "measure", "adjoint", "measure_sampled",
           "adjoint_real_sampled",
           "measure_cube", "adjoint_cube_real"]
