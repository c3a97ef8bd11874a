"""Preconditioned data duals (Section 3.2, Algorithm 2 v line with U_{l,b} = inverse
sampling density, U-metric l2-ball projections by forward-backward sub-iterations,
eta_l = 1 / ||U^1/2 Phi_l||^2) on the GPU against the FP64 oracle."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import nufft as nu
from oracle import pdfb as pd

from _fixtures import make_context, make_problem, rel_err, vis_to_internal

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {
    "tiny": dict(name="tiny", n=32, L=2, m_abs=600),
    "faceted": dict(name="faceted", n=128, L=4, Q=2, m_ratio=0.6, B=2),
}


def _run(ctx, prob, n_iter):
    X = torch.zeros((prob.L, prob.n1, prob.n2), device="cuda")
    it = [{"X": X, "Xcheck": torch.zeros_like(X), "y": vis_to_internal(ctx, torch, prob.y),
           "state": ctx.new_state(0)}]
    stats = ctx.fhs_pdfb_iter(it, n_iter)
    return it, stats


@pytest.mark.parametrize("case", list(CASES))
def test_preconditioned_pdfb_matches_oracle(case):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    kw = dict(CASES[case])
    spec, inp, prob = make_problem(kw.pop("name"), **kw)
    pd.precondition(prob, n_sub=20, power_iters=60)
    ctx = make_context(prob, torch)
    ctx.fhs_set_preconditioning(0, 20)                     # the library's own density
    # ||U^1/2 Phi_l||^2 by the library's power method: the oracle's (60 iterations) is a
    # lower bound; on the tiny case, the dense operator's largest singular value
    opn = ctx.fhs_opnorm_sq(0, 500, 1e-12)
    assert np.all(opn >= (1.0 / prob.eta) * (1 - 1e-4))
    if case == "tiny":
        for l, sl in enumerate(prob.channel_slices()):
            cols = []
            for i in range(prob.n1 * prob.n2):
                e = np.zeros(prob.n1 * prob.n2)
                e[i] = 1.0
                cols.append(np.sqrt(prob.U[sl]) * nu.measure(e.reshape(prob.n1, prob.n2), prob.uv[sl]))
            A = np.array(cols).T
            ref = np.linalg.svd(np.vstack([A.real, A.imag]), compute_uv=False)[0] ** 2
            assert opn[l] == pytest.approx(ref, rel=1e-4)
    ctx.fhs_set_params(0, prob.tau, prob.zeta, prob.kappa, prob.eta, prob.mu, prob.mu_bar, prob.eps)
    n_iter = 8
    it, stats = _run(ctx, prob, n_iter)
    st = pd.initial_state(prob)
    for _ in range(n_iter):
        out = pd.pdfb_iteration(prob, st)
    assert rel_err(it[0]["X"].double().cpu().numpy(), st.X) < 1e-4
    vu = torch.empty_like(it[0]["state"]["v"])
    ctx.fhs_vis_to_user(0, it[0]["state"]["v"], vu)
    assert rel_err(vu.cpu().numpy(), st.v) < 1e-4
    assert stats[0]["xi"] == pytest.approx(out["xi"], rel=1e-3)
    # the caller's U (the oracle's, in the caller's order) gives the same iterates bit for bit
    ctx.fhs_set_preconditioning(0, 20, prob.U.astype(np.float32))
    it2, _ = _run(ctx, prob, n_iter)
    assert torch.equal(it[0]["X"], it2[0]["X"])
    # n_sub = 0: back to the Euclidean projections of the plain method
    ctx.fhs_set_preconditioning(0, 0)
    ctx.fhs_set_params(0, prob.tau, prob.zeta, prob.kappa, np.full(prob.L, 1e-3), prob.mu, prob.mu_bar, prob.eps)
    it3, _ = _run(ctx, prob, 2)
    prob.U, prob.eta = None, np.full(prob.L, 1e-3)
    st3 = pd.initial_state(prob)
    for _ in range(2):
        pd.pdfb_iteration(prob, st3)
    assert rel_err(it3[0]["X"].double().cpu().numpy(), st3.X) < 1e-4
    ctx.close()
