"""Pins of the DDE-extended de-gridding oracle (Section 2.1, after Eq. 1) against what
the mathematics fixes, independently of its own formulas:

* the physical model: visibilities of the sky multiplied by each visibility's DDE
  pattern, by brute-force direct DFT, agree with the extended-kernel NUFFT within the
  Kaiser-Bessel interpolation accuracy;
* a one-coefficient kernel at the centre is the plain 7 x 7 Kaiser-Bessel operator;
  one at offset j is that operator at the uv point shifted by j grid cells (shift
  theorem: pins which index runs along rows and the sign of the shift);
* the adjoint is the exact transpose;
* the synthetic baseline kernels are the Fourier representation of D_a conj(D_b).
"""
from __future__ import annotations

import numpy as np
import pytest

import fhs_synth as fs
from oracle import dde
from oracle import nufft as nu


def _rand_uv(rng, M, lim=2.5):
    return rng.uniform(-lim, lim, size=(M, 2))


def test_centre_delta_is_plain_kaiser_bessel():
    rng = np.random.default_rng(1)
    K = 48
    grid = rng.standard_normal((K, K)) + 1j * rng.standard_normal((K, K))
    uv = _rand_uv(rng, 40)
    for S_d in (1, 3, 9):
        kern = np.zeros((1, S_d, S_d), dtype=complex)
        kern[0, S_d // 2, S_d // 2] = 1.0
        kidx = np.zeros(40, dtype=int)
        np.testing.assert_allclose(dde.degrid(grid, uv, kern, kidx), nu.degrid(grid, uv), rtol=0, atol=1e-12)
        v = rng.standard_normal(40) + 1j * rng.standard_normal(40)
        np.testing.assert_allclose(dde.grid_adjoint(v, uv, kern, kidx, K, K), nu.grid_adjoint(v, uv, K, K),
                                   rtol=0, atol=1e-12)


@pytest.mark.parametrize("j", [(1, 0), (0, 1), (-2, 3), (4, -4)])
def test_offset_delta_is_shifted_uv(j):
    """K = delta at (j_r, j_c): g_m[k] = phi(t + j - k), the plain row at t + j."""
    rng = np.random.default_rng(2)
    K1, K2 = 40, 56
    grid = rng.standard_normal((K1, K2)) + 1j * rng.standard_normal((K1, K2))
    uv = _rand_uv(rng, 30)
    S_d = 9
    kern = np.zeros((1, S_d, S_d), dtype=complex)
    kern[0, 4 + j[0], 4 + j[1]] = 1.0
    shifted = uv + np.array([2 * np.pi * j[1] / K2, 2 * np.pi * j[0] / K1])
    np.testing.assert_allclose(dde.degrid(grid, uv, kern, np.zeros(30, int)), nu.degrid(grid, shifted),
                               rtol=0, atol=1e-11)


def test_adjoint_is_exact_transpose():
    rng = np.random.default_rng(3)
    K1, K2, M, S_d = 32, 24, 50, 7
    kern = rng.standard_normal((5, S_d, S_d)) + 1j * rng.standard_normal((5, S_d, S_d))
    kidx = rng.integers(0, 5, M)
    uv = _rand_uv(rng, M, 3.0)
    g = rng.standard_normal((K1, K2)) + 1j * rng.standard_normal((K1, K2))
    v = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    lhs = np.vdot(v, dde.degrid(g, uv, kern, kidx))
    rhs = np.vdot(dde.grid_adjoint(v, uv, kern, kidx, K1, K2), g)
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    # image-domain pairing <Phi x, v> = <x, Phi^dagger v> (complex x)
    n1, n2 = K1 // 2, K2 // 2
    x = rng.standard_normal((n1, n2))
    lhs = np.vdot(v, dde.measure(x, uv, kern, kidx))
    rhs = np.vdot(dde.adjoint(v, uv, kern, kidx, n1, n2), x)
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))


def test_extended_nufft_matches_modulated_sky_dft():
    """The extended rows approximate the visibilities of the DDE-modulated sky to the
    accuracy of the plain 7 x 7 Kaiser-Bessel NUFFT (about 1e-6 relative here)."""
    spec = fs.CubeSpec("dde-pin", n=24, L=2, m_abs=60, B=1, n_blobs=5, seed=11)
    inp = fs.make_inputs(spec)
    dd = fs.dde_inputs(inp, n_ant=4)
    x = inp.x_true[0]
    uv = inp.uv[:60].astype(np.float64)
    kidx = dd.kidx[:60]
    got = dde.measure(x, uv, dd.kern, kidx)
    ref = dde.modulated_dft(x, uv, dd.kern, kidx)
    plain_err = np.abs(nu.measure(x, uv) - nu.direct_dft(x, uv)).max() / np.abs(nu.direct_dft(x, uv)).max()
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < 1e-5
    assert err < 20 * plain_err + 1e-12
    # the DDEs matter: the unmodulated sky is far away
    assert np.abs(nu.direct_dft(x, uv) - ref).max() / np.abs(ref).max() > 1e-2


def test_synthetic_baseline_kernels_represent_antenna_products():
    """kern[i * n_bl + k] is the Fourier representation of D_a conj(D_b): evaluating
    both sides as patterns on the pixel lattice gives the same function."""
    spec = fs.CubeSpec("dde-ant", n=16, L=2, m_abs=20, B=1, n_blobs=3, seed=5)
    inp = fs.make_inputs(spec)
    dd = fs.dde_inputs(inp, n_ant=3, S_a=3)
    rng = np.random.default_rng(spec.seed + 7919)
    rng.integers(0, 3, size=spec.M)
    n, K = spec.n, 2 * spec.n
    p = nu.pixel_coords(n)
    Ra = dd.S_a // 2
    ja = np.arange(-Ra, Ra + 1)
    taper = 0.05 * np.exp(-(ja[:, None] ** 2 + ja[None, :] ** 2) / 2.0)
    ea = np.exp(-2j * np.pi * np.outer(ja, p) / K)
    S_d = dd.kern.shape[1]
    jd = np.arange(-(S_d // 2), S_d // 2 + 1)
    ed = np.exp(-2j * np.pi * np.outer(jd, p) / K)
    pairs = [(a, b) for a in range(3) for b in range(a + 1, 3)]
    for l in range(spec.L):
        d = rng.standard_normal((3, dd.S_a, dd.S_a, 2))
        d = (d[..., 0] + 1j * d[..., 1]) * taper
        d[:, Ra, Ra] = 1.0
        D = [np.einsum("ij,ir,jc->rc", d[a], ea, ea) for a in range(3)]
        for k, (a, b) in enumerate(pairs):
            pat = np.einsum("ij,ir,jc->rc", dd.kern[l * len(pairs) + k], ed, ed)
            np.testing.assert_allclose(pat, D[a] * np.conj(D[b]), rtol=0, atol=1e-12)
