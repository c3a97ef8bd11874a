"""Parity of every libfhs operator (through the C ABI) with the FP64 oracle on
the same seeded inputs.  Bar: relative error <= 1e-5 (normwise) per operator
for the FP32 path, and element-wise |gpu - oracle| <= 1e-5 * max|oracle| + a
floor; end to end, the reconstruction SNR within 0.05 dB."""
import math

import numpy as np
import pytest

from oracle import nufft as nu
from oracle import pdfb as pd
from oracle import prox as px
from oracle import wavelets as wv
from tests._fixtures import (REL_TOL, make_context, make_problem, rel_err, to_dev_c64, to_dev_f32,
                             vis_to_internal, vis_to_user)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

CASES = {
    # tiny: 64x64, L=4, Q=1 ; faceted: 256x256, L=20, 4x4 facets, sine overlap, 2 blocks
    "tiny": dict(name="tiny"),
    "faceted": dict(name="faceted", L=6),
    "nonsquare_ragged": dict(name="faceted", n=128, L=3, Q=3, m_ratio=0.37, B=3),
    # dense coverage (about 25 visibilities per grid cell at the centre): the gridder's
    # dense-tile rounding path
    "dense": dict(name="tiny", n=64, L=2, m_abs=40000),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    kw = dict(CASES[request.param])
    spec, inp, prob = make_problem(kw.pop("name"), **kw)
    ctx = make_context(prob, torch)
    yield request.param, spec, inp, prob, ctx
    ctx.close()


@pytest.fixture(params=["fast", "plain"])
def path(request, case):
    ctx = case[4]
    ctx.fhs_set_path(request.param)
    yield request.param
    ctx.fhs_set_path("fast")


def elementwise_ok(got, ref, tol=REL_TOL):
    got, ref = np.asarray(got), np.asarray(ref)
    return np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref)) + 1e-30


def test_measure(case, path):
    _, spec, inp, prob, ctx = case
    x = inp.x_true
    y = torch.empty(prob.uv.shape[0], dtype=torch.complex64, device="cuda")
    ctx.fhs_measure(0, to_dev_f32(torch, x), y)
    got = vis_to_user(ctx, torch, y)
    ref = nu.measure_cube(x, prob.uv, prob.M_lb.sum(axis=1))
    assert rel_err(got, ref) < REL_TOL
    assert elementwise_ok(got, ref, 4 * REL_TOL)


def test_adjoint(case, path):
    _, spec, inp, prob, ctx = case
    rng = np.random.default_rng(1)
    v = rng.standard_normal(prob.uv.shape[0]) + 1j * rng.standard_normal(prob.uv.shape[0])
    v = v.astype(np.complex64).astype(np.complex128)
    x = torch.empty((prob.L, prob.n1, prob.n2), device="cuda")
    ctx.fhs_adjoint(0, vis_to_internal(ctx, torch, v), x)
    ref = nu.adjoint_cube_real(v, prob.uv, prob.M_lb.sum(axis=1), prob.n1, prob.n2)
    got = x.cpu().numpy()
    assert rel_err(got, ref) < REL_TOL
    assert elementwise_ok(got, ref, 4 * REL_TOL)


def test_adjoint_identity_on_gpu(case, path):
    _, spec, inp, prob, ctx = case
    rng = np.random.default_rng(2)
    x = rng.standard_normal((prob.L, prob.n1, prob.n2))
    v = rng.standard_normal(prob.uv.shape[0]) + 1j * rng.standard_normal(prob.uv.shape[0])
    y = torch.empty(prob.uv.shape[0], dtype=torch.complex64, device="cuda")
    ctx.fhs_measure(0, to_dev_f32(torch, x), y)
    vi = to_dev_c64(torch, v)
    xa = torch.empty((prob.L, prob.n1, prob.n2), device="cuda")
    ctx.fhs_adjoint(0, vi, xa)
    a = np.real(np.vdot(y.cpu().numpy().astype(np.complex128), v.astype(np.complex64)))
    b = np.vdot(x.astype(np.float32).astype(np.float64), xa.cpu().numpy().astype(np.float64))
    assert abs(a - b) <= 1e-5 * abs(a)


def test_sara_analysis_and_synthesis(case):
    _, spec, inp, prob, ctx = case
    rng = np.random.default_rng(3)
    x = rng.standard_normal((prob.L, prob.n1, prob.n2)).astype(np.float32).astype(np.float64)
    I = ctx.sizes(0)["n_coef"]
    assert I == wv.n_coefficients(prob.n1, prob.n2)
    c = torch.empty((prob.L, I), device="cuda")
    ctx.fhs_sara_analysis(0, to_dev_f32(torch, x), c)
    ref = wv.sara_analysis(x)
    assert rel_err(c.cpu().numpy(), ref) < REL_TOL
    assert elementwise_ok(c.cpu().numpy(), ref, 4 * REL_TOL)
    w = rng.standard_normal((prob.L, I)).astype(np.float32).astype(np.float64)
    xs = torch.empty((prob.L, prob.n1, prob.n2), device="cuda")
    ctx.fhs_sara_synthesis(0, to_dev_f32(torch, w), xs)
    ref = wv.sara_synthesis(w, prob.n1, prob.n2)
    assert rel_err(xs.cpu().numpy(), ref) < REL_TOL


def test_prox_l21_sara_facets(case, path):
    _, spec, inp, prob, ctx = case
    rng = np.random.default_rng(4)
    I = ctx.sizes(0)["n_coef"]
    xc = inp.x_true.astype(np.float32).astype(np.float64)
    W = (0.01 * rng.standard_normal((prob.L, I))).astype(np.float32).astype(np.float64)
    theta = rng.uniform(0.05, 1.0, I).astype(np.float32).astype(np.float64)
    # A starts at a small offset: the call accumulates into A (kept small so that
    # the float32 difference A - A0 does not cancel the contribution)
    A0 = (1e-3 * rng.standard_normal((prob.L, prob.n1, prob.n2))).astype(np.float32).astype(np.float64)
    Wd, thd, Ad = to_dev_f32(torch, W), to_dev_f32(torch, theta), to_dev_f32(torch, A0)
    ctx.fhs_prox_l21_sara_facets(0, to_dev_f32(torch, xc), Wd, thd, Ad)
    Wn, As = pd.sara_step(prob, xc, W, theta)
    assert rel_err(Wd.cpu().numpy(), Wn) < REL_TOL
    assert rel_err(Ad.cpu().numpy() - A0, As) < REL_TOL


def test_prox_nuclear_facets(case):
    _, spec, inp, prob, ctx = case
    rng = np.random.default_rng(5)
    xc = inp.x_true.astype(np.float32).astype(np.float64)
    P = [(0.05 * rng.standard_normal(p.shape)).astype(np.float32).astype(np.float64)
         for p in pd.initial_state(prob).P]
    tb = np.sort(rng.uniform(0.05, 1.0, (len(prob.facets), prob.L)), axis=1).astype(np.float32).astype(np.float64)
    Pd = to_dev_f32(torch, np.concatenate([p.ravel() for p in P]))
    A0 = np.zeros((prob.L, prob.n1, prob.n2))
    Ad = to_dev_f32(torch, A0)
    ctx.fhs_prox_nuclear_facets(0, to_dev_f32(torch, xc), Pd, to_dev_f32(torch, tb), Ad)
    Pn, An = pd.nuclear_step(prob, xc, P, tb)
    ref = np.concatenate([p.ravel() for p in Pn])
    assert rel_err(Pd.cpu().numpy(), ref) < REL_TOL
    assert rel_err(Ad.cpu().numpy(), An) < REL_TOL


def test_proj_l2ball_blocks(case):
    _, spec, inp, prob, ctx = case
    rng = np.random.default_rng(6)
    M = prob.uv.shape[0]
    z = (prob.y + 0.5 * (rng.standard_normal(M) + 1j * rng.standard_normal(M)) * np.abs(prob.y).mean())
    z = z.astype(np.complex64).astype(np.complex128)
    # make one block land inside its ball (no projection) to cover both branches
    l0, b0, sl0 = prob.vis_slices()[0]
    z[sl0] = prob.y[sl0] + (z[sl0] - prob.y[sl0]) * (0.5 * prob.eps[l0, b0] / np.linalg.norm(z[sl0] - prob.y[sl0]))
    z = z.astype(np.complex64).astype(np.complex128)
    zi, yi = vis_to_internal(ctx, torch, z), vis_to_internal(ctx, torch, prob.y)
    v = torch.empty_like(zi)
    dn = ctx.fhs_proj_l2ball_blocks(0, zi, yi, v)
    got = vis_to_user(ctx, torch, v)
    ref = np.zeros_like(z)
    for (l, b, sl) in prob.vis_slices():
        ref[sl] = z[sl] - px.proj_l2ball(z[sl], prob.y[sl], prob.eps[l, b])
        assert dn[l * prob.M_lb.shape[1] + b] == pytest.approx(np.linalg.norm(z[sl] - prob.y[sl]), rel=1e-6)
    assert np.all(np.abs(got[sl0]) == 0.0)
    assert rel_err(got, ref) < REL_TOL


def test_reweight(case, path):
    _, spec, inp, prob, ctx = case
    x = inp.x_true.astype(np.float32).astype(np.float64)
    I = ctx.sizes(0)["n_coef"]
    th = torch.empty(I, device="cuda")
    tb = torch.empty((len(prob.facets), prob.L), device="cuda")
    ctx.fhs_reweight(0, to_dev_f32(torch, x), th, tb)
    th_ref, tb_ref = pd.reweight(prob, x)
    assert rel_err(th.cpu().numpy(), th_ref) < REL_TOL
    assert rel_err(tb.cpu().numpy(), tb_ref) < REL_TOL


def test_opnorm_matches_dense_svd():
    # ||Phi_l||_S^2 on real images against LAPACK on the dense operator of a tiny problem
    spec, inp, prob = make_problem("tiny", n=16, L=2, m_abs=150)
    ctx = make_context(prob, torch)
    got = ctx.fhs_opnorm_sq(0, 5000, 1e-12)
    off = 0
    for l in range(prob.L):
        m = int(prob.M_lb[l].sum())
        uv = prob.uv[off:off + m]
        off += m
        cols = []
        for i in range(prob.n1 * prob.n2):
            e = np.zeros(prob.n1 * prob.n2)
            e[i] = 1.0
            cols.append(nu.measure(e.reshape(prob.n1, prob.n2), uv))
        Phi = np.array(cols).T
        ref = np.linalg.svd(np.vstack([Phi.real, Phi.imag]), compute_uv=False)[0] ** 2
        assert got[l] == pytest.approx(ref, rel=1e-4)
    ctx.close()


def _gpu_iterate(ctx, prob, n_iter, reweight_after=None, n_after=0):
    L, n1, n2 = prob.L, prob.n1, prob.n2
    X = torch.zeros((L, n1, n2), device="cuda")
    Xc = torch.zeros_like(X)
    st = ctx.new_state(0)
    y = vis_to_internal(ctx, torch, prob.y)
    it = [{"X": X, "Xcheck": Xc, "y": y, "state": st}]
    stats = ctx.fhs_pdfb_iter(it, n_iter)
    if reweight_after is not None:
        tb = st["theta_bar"]
        ctx.fhs_reweight(0, X, st["theta"], tb)
        stats = ctx.fhs_pdfb_iter(it, n_after)
    return X.cpu().numpy(), stats, st


def _oracle_iterate(prob, n_iter, reweight_after=None, n_after=0):
    st = pd.initial_state(prob)
    for _ in range(n_iter):
        out = pd.pdfb_iteration(prob, st)
    if reweight_after is not None:
        st.theta, st.theta_bar = pd.reweight(prob, st.X)
        for _ in range(n_after):
            out = pd.pdfb_iteration(prob, st)
    return st, out


def test_pdfb_end_to_end_tiny_with_reweight():
    spec, inp, prob = make_problem("tiny")
    ctx = make_context(prob, torch)
    Xg, stats, _ = _gpu_iterate(ctx, prob, 100, reweight_after=True, n_after=100)
    st, out = _oracle_iterate(prob, 100, reweight_after=True, n_after=100)
    snr_g = pd.snr_db(inp.x_true, Xg).mean()
    snr_o = pd.snr_db(inp.x_true, st.X).mean()
    assert abs(snr_g - snr_o) <= 0.05
    assert rel_err(Xg, st.X) < 1e-3
    assert stats[0]["res_norm"] == pytest.approx(np.linalg.norm(out["res"]), rel=1e-3)
    ctx.close()


@pytest.mark.parametrize("kpath", ["fast", "plain"])
def test_pdfb_end_to_end_faceted_few_iterations(kpath):
    spec, inp, prob = make_problem("faceted", L=6)
    ctx = make_context(prob, torch)
    ctx.fhs_set_path(kpath)
    Xg, stats, stg = _gpu_iterate(ctx, prob, 5)
    st, out = _oracle_iterate(prob, 5)
    assert rel_err(Xg, st.X) < 1e-4
    assert stats[0]["xi"] == pytest.approx(out["xi"], rel=1e-3)
    assert rel_err(stg["P"].cpu().numpy(), np.concatenate([p.ravel() for p in st.P])) < 1e-4
    assert rel_err(stg["W"].cpu().numpy().reshape(prob.L, -1), st.W) < 1e-4
    ctx.close()


def test_deterministic_repeat():
    """Every reduction is in a fixed order and the gridder accumulates in integers, so
    two runs from the same state agree bit for bit."""
    spec, inp, prob = make_problem("tiny")
    ctx = make_context(prob, torch)
    a, _, _ = _gpu_iterate(ctx, prob, 10)
    b, _, _ = _gpu_iterate(ctx, prob, 10)
    assert np.array_equal(a, b)
    ctx.close()


def test_kernel_timer():
    """The gridding / degridding timers record one event pair per cube inside the graph."""
    spec, inp, prob = make_problem("tiny")
    ctx = make_context(prob, torch)
    with pytest.raises(Exception):
        ctx.fhs_kernel_timer_read()
    ctx.fhs_set_kernel_timer("grid")
    _gpu_iterate(ctx, prob, 2)
    ms, n = ctx.fhs_kernel_timer_read()
    assert n == 1 and 0.0 < ms < 1000.0
    ctx.fhs_set_kernel_timer("degrid")
    _gpu_iterate(ctx, prob, 1)
    ms2, n2 = ctx.fhs_kernel_timer_read()
    assert n2 == 1 and 0.0 < ms2 < 1000.0
    ctx.fhs_set_kernel_timer(None)
    ctx.close()
