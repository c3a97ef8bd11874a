"""Pins of the Table 2 proximal operators, the one-sided Jacobi SVD and the
dual updates of Algorithm 2: closed forms, Moreau's identity, LAPACK SVD."""
import numpy as np
import pytest

from oracle import prox as px


def test_soft_threshold_and_moreau():
    rng = np.random.default_rng(0)
    z = rng.standard_normal(1000) * 3
    a = 0.7
    st = px.soft_threshold(z, a)
    assert np.allclose(st, np.where(z > a, z - a, np.where(z < -a, z + a, 0.0)))
    # prox_f + prox_{f*} = Id with f* the indicator of [-a, a]
    assert np.allclose(st + np.clip(z, -a, a), z, atol=1e-15)


def test_l21_rows_closed_form_and_single_channel():
    rng = np.random.default_rng(1)
    Z = rng.standard_normal((500, 6))
    alpha = rng.uniform(0, 3, 500)
    out = px.prox_l21_rows(Z, alpha)
    nz = np.linalg.norm(Z, axis=1)
    no = np.linalg.norm(out, axis=1)
    assert np.allclose(no, np.maximum(nz - alpha, 0), atol=1e-14)
    keep = no > 0
    assert np.allclose(out[keep] / no[keep, None], Z[keep] / nz[keep, None])
    # one channel: l2,1 is l1 -> soft threshold
    z1 = rng.standard_normal((300, 1))
    assert np.allclose(px.prox_l21_rows(z1, 0.4)[:, 0], px.soft_threshold(z1[:, 0], 0.4))
    # the l2,1 dual update with one channel is a clip (Moreau)
    w = rng.standard_normal((300, 1))
    d = px.dual_l21(w, z1, np.full(300, 0.4))
    assert np.allclose(d[:, 0], np.clip(w[:, 0] + z1[:, 0], -0.4, 0.4), atol=1e-15)


def test_l2ball_projection():
    rng = np.random.default_rng(2)
    y = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    eps = 2.0
    inside = y + 0.1 * (rng.standard_normal(50) + 1j * rng.standard_normal(50)) / 10
    assert np.allclose(px.proj_l2ball(inside, y, eps), inside)
    far = y + 5 * (rng.standard_normal(50) + 1j * rng.standard_normal(50))
    p = px.proj_l2ball(far, y, eps)
    assert np.linalg.norm(p - y) == pytest.approx(eps, rel=1e-14)
    assert np.allclose(px.proj_l2ball(p, y, eps), p)                      # idempotent
    # p - y is parallel to far - y (closest point on the sphere)
    d1, d2 = p - y, far - y
    assert np.allclose(d1 / np.linalg.norm(d1), d2 / np.linalg.norm(d2))
    # dual update = z - P_B(z) = (z - y)(1 - min(1, eps/||z - y||))
    v = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    ph = far - v
    z = v + ph
    exp = (z - y) * (1 - min(1.0, eps / np.linalg.norm(z - y)))
    assert np.allclose(px.dual_l2ball(v, ph, y, eps), exp, atol=1e-13)


def test_nonneg_projection():
    Z = np.array([[1 + 2j, -3 + 1j], [0.5, -0.0]])
    assert np.array_equal(px.proj_nonneg_real(Z), np.array([[1.0, 0.0], [0.5, 0.0]]))


@pytest.mark.parametrize("m,n", [(200, 8), (50, 20), (30, 30), (1000, 4)])
def test_jacobi_svd_matches_lapack(m, n):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n)) @ np.diag(np.logspace(0, -6, n)) @ rng.standard_normal((n, n))
    U, s, V = px.jacobi_svd(A)
    s_ref = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s, s_ref, rtol=1e-11, atol=1e-13 * s_ref[0])
    assert np.allclose((U * s) @ V.T, A, atol=1e-12 * s_ref[0])
    assert np.allclose(V.T @ V, np.eye(n), atol=1e-13)


def test_weighted_nuclear_prox_rank_one_and_lapack():
    rng = np.random.default_rng(4)
    u = rng.standard_normal(60)
    u /= np.linalg.norm(u)
    v = rng.standard_normal(5)
    v /= np.linalg.norm(v)
    Z = 3.0 * np.outer(u, v)
    alpha = np.array([1.25, 9, 9, 9, 9])
    assert np.allclose(px.prox_weighted_nuclear(Z, alpha), 1.75 * np.outer(u, v), atol=1e-13)
    Z = rng.standard_normal((80, 7))
    alpha = np.sort(rng.uniform(0.5, 4, 7))
    Uu, s, Vt = np.linalg.svd(Z, full_matrices=False)
    ref = (Uu * np.maximum(s - alpha, 0)) @ Vt
    assert np.allclose(px.prox_weighted_nuclear(Z, alpha), ref, atol=1e-12)
    # dual = Z - prox = U diag(min(s, alpha)) V^T
    P0 = rng.standard_normal((80, 7))
    X0 = Z - P0
    d = px.dual_nuclear(P0, X0, alpha)
    assert np.allclose(d, (Uu * np.minimum(s, alpha)) @ Vt, atol=1e-12)


def _metric_projection_closed_form(z, y, eps, U):
    """argmin_{||x - y|| <= eps} (x - z)^H U (x - z): x(lam) = (U z + lam y) / (U + lam)
    (stationarity with a multiplier lam >= 0), lam by bisection on ||x(lam) - y|| = eps."""
    if np.linalg.norm(z - y) <= eps:
        return z.copy()
    lo, hi = 0.0, 1.0
    f = lambda lam: np.linalg.norm((U * z + lam * y) / (U + lam) - y) - eps
    while f(hi) > 0:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if f(mid) > 0 else (lo, mid)
    lam = 0.5 * (lo + hi)
    return (U * z + lam * y) / (U + lam)


def test_metric_projection_reduces_and_converges():
    rng = np.random.default_rng(11)
    m = 300
    y = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    z = y + 3.0 * (rng.standard_normal(m) + 1j * rng.standard_normal(m))
    eps = 10.0
    # U = I: the Euclidean projection of Table 2 row 4
    assert np.allclose(px.proj_l2ball_metric(z, y, eps, np.ones(m), 20), px.proj_l2ball(z, y, eps), atol=1e-14)
    # inverse-density-like weights spanning two decades
    U = 1.0 / rng.integers(1, 100, m)
    ref = _metric_projection_closed_form(z, y, eps, U)
    x = px.proj_l2ball_metric(z, y, eps, U, 5000)
    assert np.linalg.norm(x - ref) <= 1e-6 * np.linalg.norm(ref - y)
    x20 = px.proj_l2ball_metric(z, y, eps, U, 20)
    assert np.linalg.norm(x20 - y) <= eps * (1 + 1e-12)                   # feasible
    # the metric distance decreases along the sub-iterations
    d = lambda a: np.real(np.vdot(a - z, U * (a - z)))
    assert d(ref) <= d(x20) + 1e-9 <= d(px.proj_l2ball(z, y, eps)) + 1e-9
    # inside the ball nothing moves; the preconditioned dual is then zero
    zin = y + 0.1 * (z - y) / np.linalg.norm(z - y)
    assert np.allclose(px.proj_l2ball_metric(zin, y, eps, U, 20), zin)
    v = px.dual_l2ball_precond(U * (zin - y), y, y, eps, U, 20)        # z = v / U + y = zin
    assert np.allclose(v, 0.0, atol=1e-12)


def test_inverse_density_by_counting():
    from oracle import pdfb as pd
    rng = np.random.default_rng(3)
    n = 8
    uv = rng.uniform(-np.pi, np.pi, (200, 2))
    U = pd.inverse_density(uv, n, n)
    K = 2 * n
    cells = [(int(np.floor(v * K / (2 * np.pi) + 0.5)) % K, int(np.floor(u * K / (2 * np.pi) + 0.5)) % K)
             for u, v in uv]
    for i, c in enumerate(cells):
        assert U[i] == 1.0 / sum(1 for d in cells if d == c)
