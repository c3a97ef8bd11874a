"""Image sides of the form 3 * 2^m (grid sides K = 2^a 3^b, the 768-pixel cubes of the
mixed-size batch): the mixed-radix (4, 2, 3) transforms, the conditional index wrap of
the interpolation kernels and the natural-order one-pass column transform, against the
FP64 oracle (Eq. 1, Algorithm 2), alone and batched with power-of-two cubes."""
from __future__ import annotations

import numpy as np
import pytest

import fhs_synth as fs
from oracle import nufft as nu
from oracle import pdfb as pd
from tests._fixtures import REL_TOL, make_context, make_problem, rel_err, to_dev_f32, vis_to_internal, vis_to_user

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

CASES = {
    # K = 192 = 3 * 64 (64-cell gridder tiles), 2 x 2 facets, 2 blocks
    "n96": dict(name="faceted", n=96, L=3, Q=2, m_ratio=0.5, B=2),
    # K = 96 = 3 * 32: one-visibility-per-few-cells coverage, one facet
    "n48": dict(name="tiny", n=48, L=2, m_abs=1500),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
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


def test_measure_and_adjoint(case, path):
    _, spec, inp, prob, ctx = case
    y = torch.empty(prob.uv.shape[0], dtype=torch.complex64, device="cuda")
    ctx.fhs_measure(0, to_dev_f32(torch, inp.x_true), y)
    ref = nu.measure_cube(inp.x_true, prob.uv, prob.M_lb.sum(axis=1))
    assert rel_err(vis_to_user(ctx, torch, y), ref) < REL_TOL
    rng = np.random.default_rng(1)
    m = prob.uv.shape[0]
    v = (rng.standard_normal(m) + 1j * rng.standard_normal(m)).astype(np.complex64).astype(np.complex128)
    x = torch.empty((prob.L, prob.n1, prob.n2), device="cuda")
    ctx.fhs_adjoint(0, vis_to_internal(ctx, torch, v), x)
    ref = nu.adjoint_cube_real(v, prob.uv, prob.M_lb.sum(axis=1), prob.n1, prob.n2)
    assert rel_err(x.cpu().numpy(), ref) < REL_TOL


def test_pdfb_iterations(case, path):
    _, spec, inp, prob, ctx = case
    X = torch.zeros((prob.L, prob.n1, prob.n2), device="cuda")
    st = ctx.new_state(0)
    it = [{"X": X, "Xcheck": torch.zeros_like(X), "y": vis_to_internal(ctx, torch, prob.y), "state": st}]
    stats = ctx.fhs_pdfb_iter(it, 5)
    ost = pd.initial_state(prob)
    for _ in range(5):
        out = pd.pdfb_iteration(prob, ost)
    assert rel_err(X.cpu().numpy(), ost.X) < 1e-4
    assert stats[0]["xi"] == pytest.approx(out["xi"], rel=1e-3)


def test_side_768():
    """The largest mixed-size cube side of the batch: K = 1536 = 3 * 512 (64-cell tiles)."""
    spec, inp, prob = make_problem("tiny", n=768, L=1, m_abs=60000, power_iters=3)
    ctx = make_context(prob, torch)
    y = torch.empty(prob.uv.shape[0], dtype=torch.complex64, device="cuda")
    ctx.fhs_measure(0, to_dev_f32(torch, inp.x_true), y)
    ref = nu.measure_cube(inp.x_true, prob.uv, prob.M_lb.sum(axis=1))
    assert rel_err(vis_to_user(ctx, torch, y), ref) < REL_TOL
    rng = np.random.default_rng(2)
    m = prob.uv.shape[0]
    v = (rng.standard_normal(m) + 1j * rng.standard_normal(m)).astype(np.complex64).astype(np.complex128)
    x = torch.empty((prob.L, prob.n1, prob.n2), device="cuda")
    ctx.fhs_adjoint(0, vis_to_internal(ctx, torch, v), x)
    ref = nu.adjoint_cube_real(v, prob.uv, prob.M_lb.sum(axis=1), prob.n1, prob.n2)
    assert rel_err(x.cpu().numpy(), ref) < REL_TOL
    ctx.close()


def test_batch_of_mixed_sides():
    """Cubes of sides 96, 64, 48 and 128 in one context (the twiddle table spans the
    least common multiple of the grid sides), two lanes: every cube matches its own
    oracle run."""
    from paper_2003_07358_gb300.fhs import Context, CubeParams
    shapes = [(96, 3, 2, 0.5, 2, 41), (64, 2, 1, 1.0, 1, 42), (48, 2, 1, 1.0, 2, 43), (128, 2, 2, 0.3, 1, 44)]
    probs = []
    for n, L, Q, mr, B, seed in shapes:
        spec = fs.CubeSpec(f"mixed n={n}", n=n, L=L, C=1, Q=Q, overlap=0.1, window="triangular", m_ratio=mr, B=B,
                           isnr_db=40.0, n_blobs=6, seed=seed)
        prob, _ = pd.build_problem(fs.make_inputs(spec), power_iters=20)
        prob.y = prob.y.astype(np.complex64).astype(np.complex128)
        probs.append(prob)
    ctx = Context([CubeParams(n1=p.n1, n2=p.n2, L=p.L, Qy=p.Qy, Qx=p.Qx, overlap=p.rho, window=p.window,
                              M_lb=p.M_lb, uv=p.uv, eta=p.eta, mu=p.mu, mu_bar=p.mu_bar, eps=p.eps, tau=p.tau,
                              zeta=p.zeta, kappa=p.kappa) for p in probs])
    ctx.fhs_set_lanes(2)
    its = []
    for c, p in enumerate(probs):
        X = torch.zeros((p.L, p.n1, p.n2), device="cuda")
        u = torch.as_tensor(np.ascontiguousarray(p.y, dtype=np.complex64), device="cuda")
        y = torch.empty_like(u)
        ctx.fhs_vis_to_internal(c, u, y)
        its.append({"X": X, "Xcheck": torch.zeros_like(X), "y": y, "state": ctx.new_state(c)})
    ctx.fhs_pdfb_iter(its, 3, want_stats=False)
    assert ctx.fhs_get_lanes() == 2
    for c, p in enumerate(probs):
        st = pd.initial_state(p)
        for _ in range(3):
            pd.pdfb_iteration(p, st)
        assert rel_err(its[c]["X"].cpu().numpy(), st.X) < 1e-4, c
    ctx.close()
