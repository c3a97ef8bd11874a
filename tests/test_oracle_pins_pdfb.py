"""Pins of the faceted nuclear step, the reweighting weights and the data step of the
oracle that do not go through the oracle's own formulas:

* the nuclear facet operator X -> (D_q S~_q X)_q and the primal contribution
  sum_q S~_q^T D_q P_q are adjoint to each other for Q >= 2 (Section 2.4.2, Algorithm 2
  P update and aggregation line), for both windows and ragged tiles;
* a hand-derived 12 x 12 case fixes the facet rows, the overlap and the window values;
* a facet with planted singular values gives the dual U diag(min(s, alpha)) V^T of
  Table 2 row 2 and the weights of Eq. 9 in closed form (descending pairing);
* Eq. 10 on a cube whose channels are multiples of one image: the Dirac rows have known
  norms, so the norm is taken across channels;
* the data dual uses 2 Phi x^(p) - Phi x^(p-1) = Phi (2 x^(p) - x^(p-1)) (Algorithm 2
  v line, by linearity);
* PDFB with fixed weights reaches the same point from two initialisations (a convex
  problem, Section 3.2).
"""
import math

import numpy as np
import pytest

import fhs_synth as fs
from oracle import facets as fc
from oracle import nufft as nu
from oracle import pdfb as pd
from oracle import prox as px
from oracle import wavelets as wv

HUGE = 1e30     # mu_bar so large that the prox is 0 and the dual is the identity


def _problem(n, Q, L, rho, window, mu_bar):
    """A Problem without data (the nuclear step does not read it)."""
    facets = fc.nuclear_facets(n, n, Q, Q, rho, window)
    return pd.Problem(n1=n, n2=n, L=L, Qy=Q, Qx=Q, rho=rho, window=window,
                      uv=np.zeros((L, 2)), M_lb=np.ones((L, 1), dtype=np.int64), y=np.zeros(L, complex),
                      eps=np.ones((L, 1)), eta=np.ones(L), mu=1.0, mu_bar=np.full(Q * Q, mu_bar), facets=facets)


def _zeros_like_facets(prob):
    return [np.zeros((prob.L, f["rows"][1] - f["rows"][0], f["cols"][1] - f["cols"][0])) for f in prob.facets]


@pytest.mark.parametrize("window", ["triangular", "sine"])
@pytest.mark.parametrize("n,Q,rho", [(48, 2, 0.25), (70, 3, 0.1), (64, 4, 0.3)])
def test_nuclear_facet_operator_adjoint_identity(window, n, Q, rho):
    L = 3
    prob = _problem(n, Q, L, rho, window, HUGE)
    rng = np.random.default_rng(n + Q)
    X = rng.standard_normal((L, n, n))
    G = [rng.standard_normal(p.shape) for p in _zeros_like_facets(prob)]
    tb = np.ones((Q * Q, L))
    # with an infinite threshold the dual update is Z = P + D S~ X itself
    FX, _ = pd.nuclear_step(prob, X, _zeros_like_facets(prob), tb)
    P = [g - f for g, f in zip(G, FX)]
    Pn, A = pd.nuclear_step(prob, np.zeros_like(X), G, tb)
    for a, b in zip(Pn, G):
        assert np.allclose(a, b, atol=1e-12)
    lhs = sum(float(np.vdot(f, g)) for f, g in zip(FX, G))      # <D S~ X, G>
    rhs = float(np.vdot(X, A)) / prob.zeta                      # <X, sum_q S~^T D G>
    assert lhs == pytest.approx(rhs, rel=1e-12)
    # and the same through a dual update whose input P is not zero
    Pn2, _ = pd.nuclear_step(prob, X, P, tb)
    for a, b in zip(Pn2, G):
        assert np.allclose(a, b, atol=1e-12)


def test_nuclear_facets_hand_derived_12x12():
    # n = 12, Q = 2, rho = 0.25: tiles [0, 6) and [6, 12); the second facet extends its
    # tile by floor(0.25 * 6) = 1 pixel up / left, so facets cover [0, 6) and [5, 12);
    # triangular window on an overlap of 1: w(0) = 1/2 in the later facet, 1 - 1/2 in the
    # earlier one; elsewhere 1.
    prob = _problem(12, 2, 1, 0.25, "triangular", HUGE)
    rows = [f["rows"] for f in prob.facets]
    cols = [f["cols"] for f in prob.facets]
    assert rows == [(0, 6), (0, 6), (5, 12), (5, 12)]
    assert cols == [(0, 6), (5, 12), (0, 6), (5, 12)]
    X = np.ones((1, 12, 12))
    FX, A = pd.nuclear_step(prob, X, _zeros_like_facets(prob), np.ones((4, 1)))
    w_first = np.array([1, 1, 1, 1, 1, 0.5])            # facet 0 along an axis
    w_second = np.array([0.5, 1, 1, 1, 1, 1, 1])        # facet 1 along an axis
    assert np.allclose(FX[0][0], np.outer(w_first, w_first))
    assert np.allclose(FX[3][0], np.outer(w_second, w_second))
    assert np.allclose(FX[1][0], np.outer(w_first, w_second))
    # A = sum_q D_q^2 (P = D X with X = 1): 1 away from the overlap, 1/4 + 1/4 on the
    # overlap row or column, (1/4 + 1/4)^2 where both overlaps meet
    a1 = np.ones(12)
    a1[5] = 0.5
    assert np.allclose(A[0], np.outer(a1, a1))


def _planted_facet(prob, q, s, rng):
    """X (zero outside facet q) with D_q S~_q X = U diag(s) V^T for random U, V."""
    f = prob.facets[q]
    (r0, r1), (c0, c1), D = f["rows"], f["cols"], f["D"]
    L = prob.L
    Nq = (r1 - r0) * (c1 - c0)
    U, _ = np.linalg.qr(rng.standard_normal((Nq, L)))
    V, _ = np.linalg.qr(rng.standard_normal((L, L)))
    Z = (U * s) @ V.T                                   # [pixels][channels]
    X = np.zeros((L, prob.n1, prob.n2))
    X[:, r0:r1, c0:c1] = Z.T.reshape(L, r1 - r0, c1 - c0) / D
    return X, U, V


@pytest.mark.parametrize("window,q", [("sine", 3), ("triangular", 1), ("triangular", 8)])
def test_planted_singular_values_nuclear_dual_and_weights(window, q):
    Q, L = 3, 4
    prob = _problem(60, Q, L, 0.2, window, 1.0)
    prob.mu_bar = np.linspace(0.5, 1.5, Q * Q)
    rng = np.random.default_rng(q)
    s = np.array([6.0, 2.5, 0.9, 0.05])
    X, U, V = _planted_facet(prob, q, s, rng)
    tb = np.tile(np.array([0.1, 0.6, 0.8, 1.0]), (Q * Q, 1))
    Pn, _ = pd.nuclear_step(prob, X, _zeros_like_facets(prob), tb)
    alpha = prob.mu_bar[q] / prob.zeta * tb[q]
    expect = (U * np.minimum(s, alpha)) @ V.T           # Table 2 row 2, dual form
    got = Pn[q].reshape(L, -1).T
    assert np.allclose(got, expect, atol=1e-12)
    # Eq. 9 weights, paired with the singular values in descending order
    _, tbar = pd.reweight(prob, X)
    assert np.allclose(tbar[q], prob.mu_bar[q] / (s + prob.mu_bar[q]), rtol=1e-12)


def test_eq10_weights_are_norms_across_channels():
    n, L = 32, 3
    rng = np.random.default_rng(10)
    a = rng.random((n, n)) ** 3
    c = np.array([1.0, -2.0, 0.5])
    X = c[:, None, None] * a[None]                      # channel l = c_l a
    prob = _problem(n, 1, L, 0.1, "triangular", 1.0)
    prob.mu = 0.7
    theta, _ = pd.reweight(prob, X)
    table, total = wv.coefficient_map(n, n)
    off, r, cc = table[(8, 0, 0)]                       # the Dirac block, Psi^dagger = x / 3
    dirac = theta[off:off + r * cc].reshape(r, cc)
    expect = prob.mu / (np.abs(a) * np.linalg.norm(c) / 3.0 + prob.mu)
    assert np.allclose(dirac, expect, rtol=1e-13)
    # every other row: |[Psi^dagger a]_i| ||c||
    ca = wv.sara_analysis(a[None])[0]
    assert np.allclose(theta, prob.mu / (np.abs(ca) * np.linalg.norm(c) + prob.mu), rtol=1e-12)


def test_data_dual_uses_the_extrapolated_point():
    spec = fs.workload("tiny", n=16, L=2, m_abs=120, B=2)
    inp = fs.make_inputs(spec)
    prob, _ = pd.build_problem(inp, power_iters=30)
    rng = np.random.default_rng(4)
    X_prev = rng.random((prob.L, 16, 16))
    X = rng.random((prob.L, 16, 16))
    v = (rng.standard_normal(prob.y.size) + 1j * rng.standard_normal(prob.y.size)) * 0.1
    u_prev = pd.measure_all(prob, X_prev)
    vn, u, res, A = pd.data_step(prob, X, v, u_prev)
    z = v + pd.measure_all(prob, 2.0 * X - X_prev)
    for (l, b, sl) in prob.vis_slices():
        d = z[sl] - prob.y[sl]
        nd = np.linalg.norm(d)
        expect = d * max(0.0, 1.0 - prob.eps[l, b] / nd)
        assert np.allclose(vn[sl], expect, atol=1e-12 * np.abs(d).max())
        assert res[l, b] == pytest.approx(np.linalg.norm(prob.y[sl] - pd.measure_all(prob, X)[sl]), rel=1e-12)
    assert np.allclose(u, pd.measure_all(prob, X))


@pytest.mark.slow
def test_pdfb_reaches_the_same_point_from_two_initialisations():
    spec = fs.workload("tiny", n=16, L=2, m_abs=200)
    inp = fs.make_inputs(spec)
    prob, _ = pd.build_problem(inp, power_iters=60)
    rng = np.random.default_rng(9)
    runs = []
    for X0 in (None, rng.random((2, 16, 16)) * inp.x_true.max()):
        st = pd.initial_state(prob, X0)
        for _ in range(400):
            pd.pdfb_iteration(prob, st)
        runs.append(st.X)
    assert np.linalg.norm(runs[0] - runs[1]) <= 1e-4 * np.linalg.norm(runs[0])


def test_solve_follows_the_stopping_rules():
    """Algorithm 1 around Algorithm 2: every cycle stops by its rule (p_max, or p >= p_min
    with xi and ||r|| below their bounds), cycles stop at t_max or small xi_rw, and a cycle
    with p_min = p_max = K is K plain iterations after a weight update and a restart."""
    spec = fs.workload("tiny", n=16, L=2, m_abs=200)
    inp = fs.make_inputs(spec)
    prob, _ = pd.build_problem(inp, power_iters=60)
    st = pd.initial_state(prob)
    eps_norm = np.linalg.norm(prob.eps)
    cyc = pd.solve(prob, st, p_min=5, p_max=150, xi_pdfb=5e-3, res_factor=1.01, t_max=4, xi_reweight=2e-2)
    assert 1 <= len(cyc) <= 4
    for c in cyc:
        assert 5 <= c["iterations"] <= 150
        if c["iterations"] < 150:
            assert c["xi"] <= 5e-3 and c["res_norm"] <= 1.01 * eps_norm
    assert len(cyc) == 4 or cyc[-1]["xi_rw"] <= 2e-2
    assert all(c["xi_rw"] > 2e-2 for c in cyc[:-1])
    assert cyc[0]["xi_rw"] == math.inf                 # X^(0) = 0
    # fixed counts: one cycle of K iterations equals reweight + restart + K iterations
    st1 = pd.initial_state(prob)
    pd.solve(prob, st1, p_min=7, p_max=7, xi_pdfb=0.0, res_factor=1.0, t_max=1, xi_reweight=0.0)
    st2 = pd.initial_state(prob)
    st2.theta, st2.theta_bar = pd.reweight(prob, st2.X)
    for _ in range(7):
        pd.pdfb_iteration(prob, st2)
    assert np.array_equal(st1.X, st2.X)
