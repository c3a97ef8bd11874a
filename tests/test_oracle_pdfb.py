"""Pins of the PDFB / reweighting oracle (Algorithms 1-2, Sections 2.4, 3, 4):
parameter formulas against library routines, the power method against a dense
SVD, the Q = 1 reduction to HyperSARA, and convergence properties."""
import math

import numpy as np
import pytest
from scipy import stats

import fhs_synth as fs
from oracle import facets as fc
from oracle import nufft as nu
from oracle import pdfb as pd
from oracle import prox as px
from oracle import wavelets as wv


def test_chi_moments_match_scipy():
    for k in (1, 4, 16, 20, 64):
        m, s = pd.chi_mean_std(k)
        assert m == pytest.approx(stats.chi(k).mean(), rel=1e-12)
        assert s == pytest.approx(stats.chi(k).std(), rel=1e-10)


def test_l2_radii_formula():
    eps = pd.l2_radii(0.5, [300, 700])
    e2 = 0.25 * (1000 + 2 * math.sqrt(1000))
    assert np.allclose(eps ** 2, [e2 * 0.3, e2 * 0.7])
    assert np.sum(eps ** 2) == pytest.approx(e2)


def test_noise_sigma_recovers_isnr():
    rng = np.random.default_rng(0)
    clean = rng.standard_normal(4000) + 1j * rng.standard_normal(4000)
    s = pd.noise_sigma(clean, 30.0)
    assert 10 * math.log10(np.sum(np.abs(clean) ** 2) / (4000 * s * s)) == pytest.approx(30.0)


def test_power_method_matches_dense_svd():
    rng = np.random.default_rng(1)
    n, M = 8, 40
    uv = rng.uniform(-math.pi, math.pi, (M, 2))
    cols = []
    for i in range(n * n):
        e = np.zeros(n * n)
        e[i] = 1
        cols.append(nu.measure(e.reshape(n, n), uv))
    Phi = np.array(cols).T                                   # [M][n^2] complex
    real_op = np.vstack([Phi.real, Phi.imag])                # Phi on real images
    ref = np.linalg.svd(real_op, compute_uv=False)[0] ** 2
    got = pd.op_norm_sq(uv, n, n, rng.standard_normal((n, n)), max_iter=2000, rel_tol=1e-13)
    assert got == pytest.approx(ref, rel=1e-8)


def test_fhs_heuristics_formulas():
    sig = np.array([0.3, 0.4])
    opn = np.array([4.0, 16.0])
    mu, mub = pd.fhs_heuristics(sig, opn, [100, 1])
    sb = math.sqrt((0.15 ** 2 + 0.1 ** 2) / 2)
    m, s = pd.chi_mean_std(2)
    assert mu == pytest.approx(sb * (m + s))
    assert mub[0] == pytest.approx(sb * math.sqrt(100 * 2 / 2))
    assert mub[1] == pytest.approx(sb * math.sqrt(1 * 2 / 1))


@pytest.fixture(scope="module")
def tiny():
    spec = fs.workload("tiny", n=32, L=3, m_abs=600)
    inp = fs.make_inputs(spec)
    prob, aux = pd.build_problem(inp, power_iters=100)
    return inp, prob


def test_initial_weights_are_one_and_in_unit_interval(tiny):
    inp, prob = tiny
    th, tb = pd.reweight(prob, np.zeros((prob.L, prob.n1, prob.n2)))
    assert np.all(th == 1.0) and np.all(tb == 1.0)
    th, tb = pd.reweight(prob, inp.x_true)
    assert np.all((th > 0) & (th <= 1)) and np.all((tb > 0) & (tb <= 1))


def test_q1_nuclear_step_is_hypersara_svt(tiny):
    inp, prob = tiny
    rng = np.random.default_rng(2)
    Xc = rng.random((prob.L, prob.n1, prob.n2))
    P = [rng.standard_normal((prob.L, prob.n1, prob.n2))]
    tb = np.array([[1.0, 0.5, 0.2]])
    newP, A = pd.nuclear_step(prob, Xc, P, tb)
    Z = (P[0] + Xc).reshape(prob.L, -1).T
    U, s, Vt = np.linalg.svd(Z, full_matrices=False)
    alpha = prob.mu_bar[0] / prob.zeta * tb[0]
    ref = (U * np.minimum(s, alpha)) @ Vt
    assert np.allclose(newP[0].reshape(prob.L, -1).T, ref, atol=1e-11)
    assert np.allclose(A, prob.zeta * newP[0])


def test_zero_mu_bar_gives_sara_limit(tiny):
    # (C, mu_bar) = (L, 0): the nuclear duals stay zero and each channel is an
    # independent SARA problem (Section 2.4.1)
    inp, prob = tiny
    rng = np.random.default_rng(3)
    Xc = rng.random((prob.L, prob.n1, prob.n2))
    P = [np.zeros((prob.L, prob.n1, prob.n2))]
    saved = prob.mu_bar
    prob.mu_bar = np.zeros_like(saved)
    try:
        newP, A = pd.nuclear_step(prob, Xc, P, np.ones((1, prob.L)))
    finally:
        prob.mu_bar = saved
    assert np.max(np.abs(newP[0])) < 1e-12 * np.max(Xc) and np.max(np.abs(A)) < 1e-12 * np.max(Xc)


def test_pdfb_converges_to_feasible_point(tiny):
    inp, prob = tiny
    st = pd.initial_state(prob)
    xis = []
    for _ in range(300):
        out = pd.pdfb_iteration(prob, st)
        xis.append(out["xi"])
    assert xis[-1] < 1e-4
    assert np.linalg.norm(out["res"]) <= 1.01 * np.linalg.norm(prob.eps)  # stopping rule of Algorithm 2
    assert np.all(st.X >= 0)
    assert pd.snr_db(inp.x_true, st.X).mean() > 15.0
    # near a fixed point one more iteration barely moves the primal
    X = st.X.copy()
    pd.pdfb_iteration(prob, st)
    assert np.linalg.norm(st.X - X) <= 1e-4 * np.linalg.norm(X)


def test_faceted_prior_pieces_match_definitions():
    # Psi_q^+ S_q summed over facets is Psi^+ (already pinned) and the nuclear
    # contribution sum_q S~_q^T D_q P_q of constant P = 1 is the window sum = 1
    n, Q = 64, 2
    facets = fc.nuclear_facets(n, n, Q, Q, 0.25, "triangular")
    A = np.zeros((n, n))
    for f in facets:
        (r0, r1), (c0, c1), D = f["rows"], f["cols"], f["D"]
        A[r0:r1, c0:c1] += D
    assert np.allclose(A, 1.0)
