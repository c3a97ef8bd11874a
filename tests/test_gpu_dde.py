"""DDE-extended de-gridding (Section 2.1, after Eq. 1) on the GPU against the FP64
oracle (oracle.dde): Phi and Re Phi^dagger with 1 x 1, 5 x 5 and 9 x 9 kernels (7 x 7 to
15 x 15 footprints) on one-tile and 4 x 4-tile grids (footprints wrapping around the
grid edge), the adjoint pairing, bitwise-deterministic gridding, ||Phi||^2 against a
dense SVD, PDFB iterations with the extended operator, switching back to the plain
rows, and argument errors."""
from __future__ import annotations

import numpy as np
import pytest

import fhs_synth as fs
from oracle import dde
from oracle import pdfb as pd

from _fixtures import REL_TOL, make_context, rel_err, to_dev_c64, to_dev_f32, vis_to_internal, vis_to_user

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {
    "one_tile": dict(n=32, L=2, m_abs=800, B=1, n_blobs=6),
    "tiles": dict(n=128, L=3, m_ratio=0.3, B=2, n_blobs=10),
}


def _elementwise_ok(got, ref, tol):
    return bool(np.all(np.abs(np.asarray(got) - np.asarray(ref)) <= tol * np.abs(ref).max()))


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    spec = fs.CubeSpec(request.param, seed=321, **CASES[request.param])
    inp = fs.make_inputs(spec)
    prob, aux = pd.build_problem(inp, power_iters=20)
    prob.y = prob.y.astype(np.complex64).astype(np.complex128)
    ctx = make_context(prob, torch)
    yield spec, inp, prob, aux, ctx
    ctx.close()


def _kernels(inp, S_a):
    dd = fs.dde_inputs(inp, n_ant=5, S_a=S_a)
    kern = dd.kern.astype(np.complex64).astype(np.complex128)    # what the GPU holds
    return kern, dd.kidx


@pytest.mark.parametrize("S_a", [1, 3, 5])
def test_measure_and_adjoint_match_oracle(case, S_a):
    spec, inp, prob, aux, ctx = case
    kern, kidx = _kernels(inp, S_a)
    ctx.fhs_set_dde(0, kern, kidx)
    try:
        M_l = prob.M_lb.sum(axis=1)
        x = inp.x_true
        y = torch.empty(prob.uv.shape[0], dtype=torch.complex64, device="cuda")
        ctx.fhs_measure(0, to_dev_f32(torch, x), y)
        got = vis_to_user(ctx, torch, y)
        ref = dde.measure_cube(x, prob.uv, M_l, kern, kidx)
        assert rel_err(got, ref) < REL_TOL
        assert _elementwise_ok(got, ref, 4 * REL_TOL)
        rng = np.random.default_rng(5)
        v = rng.standard_normal(prob.uv.shape[0]) + 1j * rng.standard_normal(prob.uv.shape[0])
        v = v.astype(np.complex64).astype(np.complex128)
        xa = torch.empty((prob.L, prob.n1, prob.n2), device="cuda")
        ctx.fhs_adjoint(0, vis_to_internal(ctx, torch, v), xa)
        ref = dde.adjoint_cube_real(v, prob.uv, M_l, kern, kidx, prob.n1, prob.n2)
        got = xa.cpu().numpy()
        assert rel_err(got, ref) < REL_TOL
        assert _elementwise_ok(got, ref, 4 * REL_TOL)
        # the gridding is bitwise deterministic
        xb = torch.empty_like(xa)
        ctx.fhs_adjoint(0, vis_to_internal(ctx, torch, v), xb)
        assert torch.equal(xa, xb)
        # adjoint pairing through the library alone
        xr = rng.standard_normal((prob.L, prob.n1, prob.n2))
        ctx.fhs_measure(0, to_dev_f32(torch, xr), y)
        vi = to_dev_c64(torch, v)
        ctx.fhs_adjoint(0, vi, xa)
        a = np.real(np.vdot(y.cpu().numpy().astype(np.complex128), v.astype(np.complex64)))
        b = np.vdot(xr.astype(np.float32).astype(np.float64), xa.cpu().numpy().astype(np.float64))
        assert abs(a - b) <= 1e-5 * abs(a)
    finally:
        ctx.fhs_set_dde(0)


def test_plain_rows_restored_bit_for_bit(case):
    spec, inp, prob, aux, ctx = case
    x = to_dev_f32(torch, inp.x_true)
    y0 = torch.empty(prob.uv.shape[0], dtype=torch.complex64, device="cuda")
    ctx.fhs_measure(0, x, y0)
    kern, kidx = _kernels(inp, 5)
    ctx.fhs_set_dde(0, kern, kidx)
    y1 = torch.empty_like(y0)
    ctx.fhs_measure(0, x, y1)
    assert not torch.equal(y0, y1)
    ctx.fhs_set_dde(0)
    ctx.fhs_measure(0, x, y1)
    assert torch.equal(y0, y1)


def test_argument_errors(case):
    from paper_2003_07358_gb300.fhs import FhsError
    spec, inp, prob, aux, ctx = case
    kern, kidx = _kernels(inp, 3)
    with pytest.raises(FhsError, match="INVALID_ARG"):
        ctx.fhs_set_dde(0, np.zeros((2, 4, 4), np.complex64), np.zeros(prob.uv.shape[0], np.int32))
    bad = kidx.copy()
    bad[7] = kern.shape[0]
    with pytest.raises(FhsError, match="INVALID_ARG"):
        ctx.fhs_set_dde(0, kern, bad)
    # the failed calls left the plain rows in place
    y = torch.empty(prob.uv.shape[0], dtype=torch.complex64, device="cuda")
    ctx.fhs_measure(0, to_dev_f32(torch, inp.x_true), y)
    from oracle import nufft as nu
    assert rel_err(vis_to_user(ctx, torch, y), nu.measure_cube(inp.x_true, prob.uv, prob.M_lb.sum(axis=1))) < REL_TOL


def test_opnorm_matches_dense_svd():
    """||Phi||_S^2 of the extended operator (power method on the device) against the
    largest singular value of the dense real-image operator."""
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    spec = fs.CubeSpec("dde-opnorm", n=16, L=1, m_abs=150, B=1, n_blobs=3, seed=17)
    inp = fs.make_inputs(spec)
    prob, aux = pd.build_problem(inp, power_iters=10)
    kern, kidx = _kernels(inp, 5)
    ctx = make_context(prob, torch)
    ctx.fhs_set_dde(0, kern, kidx)
    opn = ctx.fhs_opnorm_sq(0, 500, 1e-12)
    cols = []
    for i in range(spec.n * spec.n):
        e = np.zeros(spec.n * spec.n)
        e[i] = 1.0
        cols.append(dde.measure(e.reshape(spec.n, spec.n), prob.uv.astype(np.float64), kern, kidx))
    A = np.array(cols).T
    ref = np.linalg.svd(np.vstack([A.real, A.imag]), compute_uv=False)[0] ** 2
    assert opn[0] == pytest.approx(ref, rel=1e-4)
    ctx.close()


def test_pdfb_with_dde_matches_oracle():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    spec = fs.CubeSpec("dde-pdfb", n=64, L=3, Q=2, m_ratio=0.4, B=2, n_blobs=8, seed=44)
    inp = fs.make_inputs(spec)
    prob, aux = pd.build_problem(inp, power_iters=20)
    dd = fs.dde_inputs(inp, n_ant=6, S_a=5)
    dd.kern = dd.kern.astype(np.complex64).astype(np.complex128)
    pd.with_dde(prob, inp, dd, aux["sigma"], power_iters=40)
    prob.y = prob.y.astype(np.complex64).astype(np.complex128)
    ctx = make_context(prob, torch)
    ctx.fhs_set_dde(0, dd.kern, dd.kidx)
    X = torch.zeros((prob.L, prob.n1, prob.n2), device="cuda")
    it = [{"X": X, "Xcheck": torch.zeros_like(X), "y": vis_to_internal(ctx, torch, prob.y), "state": ctx.new_state(0)}]
    n_iter = 8
    stats = ctx.fhs_pdfb_iter(it, n_iter)
    st = pd.initial_state(prob)
    for _ in range(n_iter):
        out = pd.pdfb_iteration(prob, st)
    assert rel_err(it[0]["X"].double().cpu().numpy(), st.X) < 1e-4
    assert stats[0]["xi"] == pytest.approx(out["xi"], rel=1e-3)
    assert stats[0]["res_norm"] == pytest.approx(float(np.linalg.norm(out["res"])), rel=1e-4)
    ctx.close()
