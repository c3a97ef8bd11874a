"""Pins of the measurement-operator oracle (Eq. 1): closed forms, the direct DFT,
library quadrature and the adjoint identity."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import nufft as nu


def test_kb_kernel_special_values():
    # phi(0) = 1, phi(+-J/2) = 1 / I0(beta), zero outside, even
    assert nu.kb_kernel(np.array([0.0]))[0] == pytest.approx(1.0, abs=1e-15)
    edge = nu.kb_kernel(np.array([3.5, -3.5]))
    assert np.allclose(edge, 1.0 / np.i0(nu.BETA), rtol=1e-14)
    assert np.all(nu.kb_kernel(np.array([3.5001, -4.0, 10.0])) == 0.0)
    u = np.linspace(-3.4, 3.4, 17)
    assert np.allclose(nu.kb_kernel(u), nu.kb_kernel(-u), rtol=0, atol=0)


@pytest.mark.parametrize("theta", [0.0, 0.1, 0.5, 1.0, math.pi / 2, 2.5])
def test_kb_ft_closed_form_matches_quadrature(theta):
    q = quad(lambda u: nu.kb_kernel(np.array([u]))[0] * math.cos(theta * u), -3.5, 3.5,
             limit=400, epsabs=1e-13)[0]
    assert nu.kb_kernel_ft(np.array([theta]))[0] == pytest.approx(q, rel=1e-10)


def test_taps_cover_support():
    t = np.array([-10.3, 0.0, 0.5, 3.49, 1234.75])
    k, w = nu.taps(t)
    assert np.all(np.diff(k, axis=1) == 1)
    assert np.all(np.abs(t[:, None] - k) <= 3.5)
    assert np.all(w > 0)


@pytest.mark.parametrize("n1,n2,M", [(32, 32, 300), (64, 64, 400), (48, 32, 250), (96, 48, 300)])
def test_nufft_matches_direct_dft(n1, n2, M):
    rng = np.random.default_rng(n1 * 7 + n2)
    x = rng.random((n1, n2))
    uv = rng.uniform(-math.pi, math.pi, (M, 2)).astype(np.float32)
    yd = nu.direct_dft(x, uv)
    yn = nu.measure(x, uv)
    assert np.linalg.norm(yn - yd) / np.linalg.norm(yd) < 1e-5


def test_point_source_phase():
    # a unit impulse at centred coordinate (p_r, p_c) has visibilities exp(-i(u p_c + v p_r))
    n = 32
    x = np.zeros((n, n))
    x[20, 9] = 1.0
    uv = np.array([[0.3, -1.2], [2.0, 0.7], [-3.0, 3.0]])
    expect = np.exp(-1j * (uv[:, 0] * (9 - 16) + uv[:, 1] * (20 - 16)))
    assert np.max(np.abs(nu.measure(x, uv) - expect)) < 1e-5


def test_adjoint_identity_complex_and_real():
    rng = np.random.default_rng(3)
    n1, n2, M = 24, 40, 500
    uv = rng.uniform(-math.pi, math.pi, (M, 2))
    xc = rng.standard_normal((n1, n2)) + 1j * rng.standard_normal((n1, n2))
    v = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    # measure() is linear over complex images: zpad_fft accepts complex input
    a = np.vdot(nu.degrid(np.fft.fft2(_zpad(xc)), uv), v)
    b = np.vdot(xc, nu.adjoint(v, uv, n1, n2))
    assert abs(a - b) <= 1e-12 * abs(a)
    xr = rng.standard_normal((n1, n2))
    a = np.real(np.vdot(nu.measure(xr, uv), v))
    b = np.vdot(xr, nu.adjoint(v, uv, n1, n2).real)
    assert abs(a - b) <= 1e-12 * abs(a)


def _zpad(x):
    n1, n2 = x.shape
    K1, K2 = 2 * n1, 2 * n2
    g = np.zeros((K1, K2), dtype=np.complex128)
    s = np.outer(nu.scaling(n1, K1), nu.scaling(n2, K2))
    g[np.ix_(nu.pixel_coords(n1) % K1, nu.pixel_coords(n2) % K2)] = s * x
    return g


def test_scaling_is_inverse_kernel_transform():
    s = nu.scaling(64, 128)
    p = nu.pixel_coords(64)
    assert np.allclose(s * nu.kb_kernel_ft(2 * np.pi * p / 128), 1.0, rtol=1e-14)
    assert np.all(s > 0)


@pytest.mark.parametrize("n1,n2", [(16, 16), (12, 20)])
def test_sampled_measure_matches_fft_route_and_direct_dft(n1, n2):
    """The FFT-free sampled evaluation equals G F Z x (numpy.fft route) to rounding and
    the exact direct DFT to the interpolation error (Eq. 1)."""
    rng = np.random.default_rng(11)
    x = rng.random((n1, n2))
    uv = rng.uniform(-np.pi, np.pi, size=(40, 2))
    ys = nu.measure_sampled(x, uv)
    yf = nu.measure(x, uv)
    assert np.abs(ys - yf).max() <= 1e-11 * np.abs(yf).max()
    yd = nu.direct_dft(x, uv)
    assert np.linalg.norm(ys - yd) <= 1e-3 * np.linalg.norm(yd)


def test_sampled_adjoint_matches_fft_route():
    """Direct per-pixel summation of Re Phi^dagger v equals the gridding + inverse FFT route."""
    rng = np.random.default_rng(12)
    n1, n2 = 14, 18
    uv = rng.uniform(-np.pi, np.pi, size=(60, 2))
    v = rng.standard_normal(60) + 1j * rng.standard_normal(60)
    full = nu.adjoint(v, uv, n1, n2).real
    pix = [(0, 0), (3, 17), (13, 5), (7, 9)]
    got = nu.adjoint_real_sampled(v, uv, n1, n2, pix)
    want = np.array([full[r, c] for r, c in pix])
    assert np.abs(got - want).max() <= 1e-11 * np.abs(full).max()
