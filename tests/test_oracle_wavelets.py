"""Pins of the SARA dictionary oracle (Section 2.3.1): Daubechies conditions,
textbook closed forms, perfect reconstruction Psi Psi^dagger = I, ||Psi^dagger|| = 1."""
import math

import numpy as np
import pytest

from oracle import wavelets as wv


@pytest.mark.parametrize("N", range(1, 9))
def test_daubechies_conditions(N):
    h = wv.daubechies(N)
    F = h.size
    assert F == 2 * N
    assert h.sum() == pytest.approx(math.sqrt(2.0), abs=1e-14)
    assert (h * h).sum() == pytest.approx(1.0, abs=1e-13)
    for m in range(1, N):                       # even-shift orthogonality
        assert abs(np.dot(h[:F - 2 * m], h[2 * m:])) < 1e-13
    g = wv.highpass(h)
    k = np.arange(F, dtype=np.float64)
    for p in range(N):                           # N vanishing moments
        assert abs(np.sum(g * k ** p)) <= 1e-12 * np.sum(np.abs(g) * k ** p)
    # extremal phase: roots of sum h[k] w^k other than w = -1 lie outside the unit circle
    r = np.roots(h[::-1])
    far = r[np.abs(r + 1) > 1e-2]
    assert np.all(np.abs(far) > 1.0)


def test_db1_db2_closed_forms():
    assert np.allclose(wv.daubechies(1), [1 / math.sqrt(2)] * 2, atol=1e-16)
    s3 = math.sqrt(3.0)
    db2 = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * math.sqrt(2))
    assert np.allclose(wv.daubechies(2), db2, atol=1e-15)


def test_haar_level_by_hand():
    a = np.array([[1.0, 2.0, 3.0, 4.0]])
    h = wv.daubechies(1)
    lo = wv.analysis_1d(a, h, -1)
    hi = wv.analysis_1d(a, wv.highpass(h), -1)
    r2 = math.sqrt(2)
    # c[k] = h0 a[2k+1] + h1 a[2k]; g = (h1, -h0) -> g0 a[2k+1] + g1 a[2k]
    assert np.allclose(lo, [[3 / r2, 7 / r2]])
    assert np.allclose(hi, [[1 / r2, 1 / r2]])


def test_level_sizes_rule():
    s = wv.level_sizes(4096, 4096, 16)
    assert s[1:] == [(2055, 2055), (1035, 1035), (525, 525), (270, 270)]


@pytest.mark.parametrize("shape", [(37, 50), (64, 64), (16, 24)])
def test_perfect_reconstruction_isometry_adjoint(shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal((2,) + shape)
    c = wv.sara_analysis(x)
    assert c.shape[-1] == wv.n_coefficients(*shape)
    assert np.max(np.abs(wv.sara_synthesis(c, *shape) - x)) < 1e-12        # Psi Psi^+ = I
    assert np.linalg.norm(c) == pytest.approx(np.linalg.norm(x), rel=1e-13)  # ||Psi^+ x|| = ||x||
    w = rng.standard_normal(c.shape)
    assert np.vdot(c, w) == pytest.approx(np.vdot(x, wv.sara_synthesis(w, *shape)), rel=1e-12)


def test_single_basis_isometry_and_dirac_block():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((20, 28))
    for N in (1, 4, 8):
        h = wv.daubechies(N)
        det, ll = wv.dwt2(x, h)
        e = sum(np.sum(d * d) for trio in det for d in trio) + np.sum(ll * ll)
        assert e == pytest.approx(np.sum(x * x), rel=1e-13)
        assert np.allclose(wv.idwt2(det, ll, h, 20, 28), x, atol=1e-12)
    table, total = wv.coefficient_map(20, 28)
    off, r, c = table[(8, 0, 0)]
    assert np.allclose(wv.sara_analysis(x)[off:off + r * c], x.ravel() / 3.0)
    assert total == wv.n_coefficients(20, 28)
