"""Operator parity at the precision workload (1024 x 1024, L = 32, 8 x 8 facets, M = N
in 4 blocks) and on one sub-cube of the large workload (4096 x 4096, L_c = 16, 16 x 16
facets, M = 0.5 N in 8 blocks: the launch configuration bench.py times).

The FP64 oracle cannot run whole operators at these sizes, so it checks what it can
compute piece by piece (every check follows from the definitions, at any size):

* the l2,1 dual of the coefficients owned by three facets (corner, interior, last), from
  the facet-local analysis Psi_q^dagger S_q X (Section 2.4.2: W_q depends on facet q
  alone);
* the nuclear dual P_q of the same three facets (Table 2 row 2, Algorithm 2 P update),
  and A = zeta D_q P_q on their pixels that no other facet covers;
* the weights of Eqs. 9-10 on those facets;
* the l2-ball data duals of every block (Table 2 row 4);
* Phi at sampled visibilities and Re Phi^dagger at sampled pixels (Eq. 1);
* the first PDFB iteration from zero (Algorithm 2): P = W = 0, so
  X^(1) = max(0, tau eta Re Phi^dagger y_b (1 - eps_b / ||y_b||)) at sampled pixels.
"""
from __future__ import annotations

import numpy as np
import pytest

import fhs_synth as fs
from oracle import facets as fc
from oracle import nufft as nu
from oracle import prox as px

from _fixtures import REL_TOL, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = {
    # workload, sub-cube, mu, mu_bar, facets checked (corner, interior, last)
    "precision": dict(workload="precision", mu=0.05, mu_bar=8.0),
    "large": dict(workload="large", mu=0.05, mu_bar=12.0),
}


def _facets_to_check(Q):
    return [0, (Q // 2) * Q + Q // 2 - 1, Q * Q - 1]


@pytest.fixture(scope="module", params=list(SHAPES))
def cube(request):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2003_07358_gb300.fhs import Context, CubeParams
    cfg = SHAPES[request.param]
    spec = fs.workload(cfg["workload"])
    rng = np.random.default_rng(spec.seed)
    sources = fs.sky_sources(spec, rng)
    base = fs.base_uv(spec, rng)
    blocks = fs.radial_blocks(base, spec.B)
    perm = np.concatenate(blocks)
    chans = fs.subcube_channels(spec, 0)
    Lc, n, Q = spec.Lc, spec.n, spec.Q
    M_lb = np.array([[b.size for b in blocks]] * Lc, dtype=np.int64)
    uv = np.concatenate([fs.channel_uv(base, spec, l)[perm] for l in chans])
    eta = np.linspace(0.5, 1.5, Lc) * 1e-3
    eps = np.ones((Lc, spec.B))
    mu_bar = np.full(Q * Q, cfg["mu_bar"])
    cp = CubeParams(n1=n, n2=n, L=Lc, Qy=Q, Qx=Q, overlap=spec.overlap, window=spec.window, M_lb=M_lb, uv=uv,
                    eta=eta, mu=cfg["mu"], mu_bar=mu_bar, eps=eps)
    ctx = Context([cp])
    x = np.stack([fs.render_channel(spec, sources, int(l)).astype(np.float32) for l in chans]).astype(np.float64)
    facets = fc.nuclear_facets(n, n, Q, Q, spec.overlap, spec.window)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(spec.seed + 17)
    d = dict(name=request.param, spec=spec, ctx=ctx, x=x, xd=torch.as_tensor(x.astype(np.float32), device="cuda"),
             uv=uv, M_lb=M_lb, eta=eta, eps=eps, mu=cfg["mu"], mu_bar=mu_bar, facets=facets, gen=gen, n=n, Q=Q,
             Lc=Lc)
    yield d
    ctx.close()
    del d
    torch.cuda.empty_cache()


def _facet_offsets(facets, L):
    off, out = 0, []
    for f in facets:
        out.append(off)
        off += L * (f["rows"][1] - f["rows"][0]) * (f["cols"][1] - f["cols"][0])
    return out, off


def test_l21_dual_on_three_facets(cube):
    ctx, L, n, Q = cube["ctx"], cube["Lc"], cube["n"], cube["Q"]
    I = ctx.sizes(0)["n_coef"]
    g = cube["gen"]
    W = 0.01 * torch.randn((L, I), device="cuda", generator=g)
    theta = 0.05 + 0.95 * torch.rand(I, device="cuda", generator=g)
    A = torch.zeros((L, n, n), device="cuda")
    checks = []
    for q in _facets_to_check(Q):
        qy, qx = divmod(q, Q)
        idx, coef = fc.sara_facet_analysis_local(cube["x"], Q, Q, qy, qx)
        it = torch.as_tensor(idx, device="cuda")
        checks.append((idx, coef, W[:, it].double().cpu().numpy(), theta[it].double().cpu().numpy()))
    ctx.fhs_prox_l21_sara_facets(0, cube["xd"], W, theta, A)
    for idx, coef, W0, th in checks:
        ref = px.dual_l21(W0.T, coef.T, cube["mu"] * th).T
        got = W[:, torch.as_tensor(idx, device="cuda")].double().cpu().numpy()
        assert rel_err(got, ref) < REL_TOL
        assert np.max(np.abs(got - ref)) <= 4 * REL_TOL * np.max(np.abs(ref))
    del W, theta, A


def test_nuclear_dual_on_three_facets(cube):
    ctx, L, n, Q, facets = cube["ctx"], cube["Lc"], cube["n"], cube["Q"], cube["facets"]
    offs, total = _facet_offsets(facets, L)
    assert total == L * ctx.sizes(0)["n_facet_pix"]
    g = cube["gen"]
    P = 0.05 * torch.randn(total, device="cuda", generator=g)
    tb = np.sort(np.random.default_rng(3).uniform(0.05, 1.0, (Q * Q, L)), axis=1).astype(np.float32)
    A = torch.zeros((L, n, n), device="cuda")
    cover = np.zeros((n, n), dtype=np.int32)
    for f in facets:
        cover[f["rows"][0]:f["rows"][1], f["cols"][0]:f["cols"][1]] += 1
    before = {}
    for q in _facets_to_check(Q):
        f = facets[q]
        h, w = f["rows"][1] - f["rows"][0], f["cols"][1] - f["cols"][0]
        before[q] = P[offs[q]:offs[q] + L * h * w].double().cpu().numpy().reshape(L, h, w)
    ctx.fhs_prox_nuclear_facets(0, cube["xd"], P, torch.as_tensor(tb, device="cuda"), A)
    An = A.double().cpu().numpy()
    for q, P0 in before.items():
        f = facets[q]
        (r0, r1), (c0, c1), D = f["rows"], f["cols"], f["D"]
        h, w = r1 - r0, c1 - c0
        DX = (cube["x"][:, r0:r1, c0:c1] * D).reshape(L, -1).T
        alpha = cube["mu_bar"][q] * tb[q].astype(np.float64)
        ref = px.dual_nuclear(P0.reshape(L, -1).T, DX, alpha)                # [pixels][channels]
        got = P[offs[q]:offs[q] + L * h * w].double().cpu().numpy().reshape(L, -1).T
        assert rel_err(got, ref) < REL_TOL, q
        only = cover[r0:r1, c0:c1] == 1                     # pixels no other facet covers
        refA = (ref.T.reshape(L, h, w) * D)[:, only]
        assert rel_err(An[:, r0:r1, c0:c1][:, only], refA) < REL_TOL, q
    del P, A


def test_reweight_on_three_facets(cube):
    ctx, L, n, Q, facets = cube["ctx"], cube["Lc"], cube["n"], cube["Q"], cube["facets"]
    I = ctx.sizes(0)["n_coef"]
    th = torch.empty(I, device="cuda")
    tb = torch.empty((Q * Q, L), device="cuda")
    ctx.fhs_reweight(0, cube["xd"], th, tb)
    tbn = tb.double().cpu().numpy()
    for q in _facets_to_check(Q):
        qy, qx = divmod(q, Q)
        idx, coef = fc.sara_facet_analysis_local(cube["x"], Q, Q, qy, qx)
        ref = cube["mu"] / (np.linalg.norm(coef, axis=0) + cube["mu"])               # Eq. 10
        got = th[torch.as_tensor(idx, device="cuda")].double().cpu().numpy()
        assert rel_err(got, ref) < REL_TOL
        f = facets[q]
        (r0, r1), (c0, c1), D = f["rows"], f["cols"], f["D"]
        _, s, _ = px.jacobi_svd((cube["x"][:, r0:r1, c0:c1] * D).reshape(L, -1).T)
        ref = cube["mu_bar"][q] / (s + cube["mu_bar"][q])                           # Eq. 9
        assert rel_err(tbn[q], ref) < REL_TOL, q


def test_l2ball_duals_every_block(cube):
    ctx, L, B = cube["ctx"], cube["Lc"], cube["spec"].B
    M_lb = cube["M_lb"]
    nv = int(M_lb.sum())
    rng = np.random.default_rng(8)
    y = (rng.standard_normal(nv) + 1j * rng.standard_normal(nv)).astype(np.complex64)
    z = (y + 0.3 * (rng.standard_normal(nv) + 1j * rng.standard_normal(nv))).astype(np.complex64)
    # radii: half of the blocks end up inside their ball (no projection)
    off = np.concatenate([[0], np.cumsum(M_lb.ravel())])
    dn_ref = np.array([np.linalg.norm(z[off[k]:off[k + 1]].astype(np.complex128) - y[off[k]:off[k + 1]])
                       for k in range(L * B)])
    eps = dn_ref * np.where(np.arange(L * B) % 2 == 0, 0.5, 1.5)
    ctx.fhs_set_params(0, 0.33, 1.0, 1.0, cube["eta"], cube["mu"], cube["mu_bar"], eps)
    zi, yi = torch.empty(nv, dtype=torch.complex64, device="cuda"), torch.empty(nv, dtype=torch.complex64, device="cuda")
    ctx.fhs_vis_to_internal(0, torch.as_tensor(z, device="cuda"), zi)
    ctx.fhs_vis_to_internal(0, torch.as_tensor(y, device="cuda"), yi)
    v = torch.empty_like(zi)
    dn = ctx.fhs_proj_l2ball_blocks(0, zi, yi, v)
    vu = torch.empty_like(v)
    ctx.fhs_vis_to_user(0, v, vu)
    got = vu.cpu().numpy()
    worst = 0.0
    for k in range(L * B):
        sl = slice(off[k], off[k + 1])
        ref = px.dual_l2ball(np.zeros(off[k + 1] - off[k]), z[sl].astype(np.complex128), y[sl].astype(np.complex128),
                             eps[k])
        if k % 2:
            assert np.all(got[sl] == 0)
        else:
            worst = max(worst, rel_err(got[sl], ref))
    assert worst < REL_TOL
    assert np.allclose(dn, dn_ref, rtol=1e-6)
    ctx.fhs_set_params(0, 0.33, 1.0, 1.0, cube["eta"], cube["mu"], cube["mu_bar"], cube["eps"])


def test_measure_and_adjoint_sampled(cube):
    ctx, L, n, xd = cube["ctx"], cube["Lc"], cube["n"], cube["xd"]
    nv = int(cube["M_lb"].sum())
    Ml = int(cube["M_lb"][0].sum())
    y = torch.empty(nv, dtype=torch.complex64, device="cuda")
    ctx.fhs_measure(0, xd, y)
    yu = torch.empty_like(y)
    ctx.fhs_vis_to_user(0, y, yu)
    rng = np.random.default_rng(6)
    got, want = [], []
    for l in (0, L // 2, L - 1):
        idx = np.sort(rng.choice(Ml, size=24, replace=False)) + l * Ml
        got.append(yu[torch.as_tensor(idx, device="cuda")].cpu().numpy())
        want.append(nu.measure_sampled(cube["x"][l], cube["uv"][idx]))
    assert rel_err(np.concatenate(got), np.concatenate(want)) <= REL_TOL
    out = torch.empty_like(xd)
    ctx.fhs_adjoint(0, y, out)
    l = L - 1
    img = out[l].double().cpu().numpy()
    pix = [(n // 2, n // 2), (3, n - 5), (n - 1, 0), (n // 3, 2 * n // 3)]
    v = yu[l * Ml:(l + 1) * Ml].cpu().numpy().astype(np.complex128)
    want = nu.adjoint_real_sampled(v, cube["uv"][l * Ml:(l + 1) * Ml], n, n, pix)
    assert np.abs(np.array([img[r, c] for r, c in pix]) - want).max() <= REL_TOL * np.abs(img).max()


def test_first_pdfb_iteration_primal_update_sampled(cube):
    """From X = 0 with zero duals, A = eta Re Phi^dagger v^(1) with v^(1)_b = -y_b (1 - eps_b/||y_b||)
    and X^(1) = max(0, -tau A)."""
    ctx, L, n, B = cube["ctx"], cube["Lc"], cube["n"], cube["spec"].B
    M_lb = cube["M_lb"]
    nv = int(M_lb.sum())
    Ml = int(M_lb[0].sum())
    g = cube["gen"]
    yu = torch.randn(nv, dtype=torch.complex64, device="cuda", generator=g)
    yi = torch.empty_like(yu)
    ctx.fhs_vis_to_internal(0, yu, yi)
    yh = yu.cpu().numpy().astype(np.complex128)
    off = np.concatenate([[0], np.cumsum(M_lb.ravel())])
    ynorm = np.array([np.linalg.norm(yh[off[k]:off[k + 1]]) for k in range(L * B)])
    eps = 0.9 * ynorm
    ctx.fhs_set_params(0, 0.33, 1.0, 1.0, cube["eta"], cube["mu"], cube["mu_bar"], eps)
    X = torch.zeros((L, n, n), device="cuda")
    it = [{"X": X, "Xcheck": torch.zeros_like(X), "y": yi, "state": ctx.new_state(0)}]
    st = ctx.fhs_pdfb_iter(it, 1)
    assert st[0]["res_norm"] == pytest.approx(np.linalg.norm(ynorm), rel=1e-6)
    v1 = np.zeros_like(yh)
    for k in range(L * B):
        sl = slice(off[k], off[k + 1])
        v1[sl] = px.dual_l2ball(np.zeros(off[k + 1] - off[k]), np.zeros(off[k + 1] - off[k]), yh[sl], eps[k])
    pix = [(n // 2, n // 2 + 1), (n // 2 - 7, n // 2 + 3), (1, 2), (n - 2, n // 4)]
    for l in (0, L - 1):
        sl = slice(l * Ml, (l + 1) * Ml)
        A = cube["eta"][l] * nu.adjoint_real_sampled(v1[sl], cube["uv"][sl], n, n, pix)
        ref = np.maximum(0.0, -0.33 * A)
        Xl = X[l].double().cpu().numpy()
        got = np.array([Xl[r, c] for r, c in pix])
        assert np.abs(got - ref).max() <= 4 * REL_TOL * 0.33 * np.abs(A).max(), (got, ref)
        # X^(1) >= 0 everywhere and X_check = 2 X^(1) - X^(0) = 2 X^(1)
        assert float(X[l].min()) >= 0.0
    assert torch.equal(it[0]["Xcheck"], 2 * X)
    ctx.fhs_set_params(0, 0.33, 1.0, 1.0, cube["eta"], cube["mu"], cube["mu_bar"], cube["eps"])
