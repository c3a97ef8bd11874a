"""Noise-based parameters computed on the device (fhs_heuristic_params) against the
oracle's formulas (Eq. 3 radii, FHS sparsity and low-rank heuristics, Section 2.4.2) and
its power method (Section 2.3.1 footnote)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import pdfb as pd

from _fixtures import make_context, make_problem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("over", [dict(L=6), dict(n=128, L=3, Q=3, m_ratio=0.37, B=3)])
def test_heuristic_params_match_oracle(over):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    spec, inp, prob = make_problem("faceted", power_iters=100, **over)
    ctx = make_context(prob, torch)
    sigma = np.linspace(0.5, 2.0, prob.L)                  # any noise levels
    got = ctx.fhs_heuristic_params(0, sigma, power_iters=200, rel_tol=1e-9)
    opn_gpu = 1.0 / got["eta"]
    # the power method itself (pinned against dense SVDs on tiny problems elsewhere): two
    # power methods from different start vectors agree to the slow convergence of
    # nearly equal top eigenvalues; the formulas below use the library's own norms
    assert np.allclose(opn_gpu, 1.0 / prob.eta, rtol=2e-2)
    # the formulas, evaluated by the oracle on the same operator norms
    npix = [(f["rows"][1] - f["rows"][0]) * (f["cols"][1] - f["cols"][0]) for f in prob.facets]
    mu, mu_bar = pd.fhs_heuristics(sigma, opn_gpu, npix)
    assert got["mu"] == pytest.approx(mu, rel=1e-12)
    assert np.allclose(got["mu_bar"], mu_bar, rtol=1e-12)
    for l in range(prob.L):
        assert np.allclose(got["eps"][l], pd.l2_radii(sigma[l], prob.M_lb[l]), rtol=1e-12)
    # installed in the context: a PDFB iteration with them matches the oracle's
    prob.eta, prob.mu, prob.mu_bar, prob.eps = got["eta"], got["mu"], got["mu_bar"], got["eps"]
    st = pd.initial_state(prob)
    pd.pdfb_iteration(prob, st)
    pd.pdfb_iteration(prob, st)
    X = torch.zeros((prob.L, prob.n1, prob.n2), device="cuda")
    u = torch.as_tensor(np.ascontiguousarray(prob.y, dtype=np.complex64), device="cuda")
    y = torch.empty_like(u)
    ctx.fhs_vis_to_internal(0, u, y)
    it = [{"X": X, "Xcheck": torch.zeros_like(X), "y": y, "state": ctx.new_state(0)}]
    stats = ctx.fhs_pdfb_iter(it, 2)
    assert stats[0]["eps_norm"] == pytest.approx(np.linalg.norm(prob.eps), rel=1e-12)
    err = np.linalg.norm(X.double().cpu().numpy() - st.X) / np.linalg.norm(st.X)
    assert err < 1e-4
    ctx.close()
