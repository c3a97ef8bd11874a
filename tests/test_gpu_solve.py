"""Algorithm 1 around Algorithm 2 with their stopping rules, run on the device by
fhs_solve (one graph with nested WHILE nodes per cube), against the oracle's solve.

* The cycle count and the PDFB iterations of every cycle follow the same rules: equal
  cycle counts, iteration counts within 2 (FP32 and FP64 statistics can fall on either
  side of a threshold near its crossing), reconstruction SNR within 0.05 dB.
* The SARA limit of Section 2.4.1 (C = L, mu_bar = 0): the nuclear duals stay zero.
* A NaN in the data stops both loops and is reported as NONFINITE.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import pdfb as pd

from _fixtures import make_context, make_problem, rel_err, vis_to_internal

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RULES = dict(p_min=10, p_max=120, xi_pdfb=2e-3, res_factor=1.01, t_max=3, xi_reweight=1e-2)


def _iterate(ctx, prob, y_user):
    X = torch.zeros((prob.L, prob.n1, prob.n2), device="cuda")
    return [{"X": X, "Xcheck": torch.zeros_like(X), "y": vis_to_internal(ctx, torch, y_user),
             "state": ctx.new_state(0)}]


@pytest.fixture(scope="module")
def tiny():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    spec, inp, prob = make_problem("tiny")
    return spec, inp, prob


def test_solve_matches_oracle_algorithm_1(tiny):
    spec, inp, prob = tiny
    ctx = make_context(prob, torch)
    it = _iterate(ctx, prob, prob.y)
    rep = ctx.fhs_solve(it, **RULES)[0]
    st = pd.initial_state(prob)
    cyc = pd.solve(prob, st, **RULES)
    assert rep["cycles"] == len(cyc)
    assert not rep["nonfinite"]
    for got, ref in zip(rep["iterations_per_cycle"], cyc):
        assert abs(got - ref["iterations"]) <= 2, (rep["iterations_per_cycle"], [c["iterations"] for c in cyc])
    assert rep["iterations"] == sum(rep["iterations_per_cycle"])
    Xg = it[0]["X"].double().cpu().numpy()
    assert abs(pd.snr_db(inp.x_true, Xg).mean() - pd.snr_db(inp.x_true, st.X).mean()) <= 0.05
    assert rel_err(Xg, st.X) < 1e-2
    # the last cycle stopped by a rule
    assert rep["cycles"] == RULES["t_max"] or rep["xi_reweight"] <= RULES["xi_reweight"]
    ctx.close()


def test_solve_fixed_counts_equal_plain_iterations(tiny):
    """p_min = p_max = K, one cycle: weights from X = 0 (all ones), K iterations; the same
    as fhs_pdfb_iter from the zero state, bit for bit (same kernels, same order)."""
    spec, inp, prob = tiny
    ctx = make_context(prob, torch)
    it1 = _iterate(ctx, prob, prob.y)
    u0 = torch.zeros_like(it1[0]["y"])
    rep = ctx.fhs_solve(it1, p_min=7, p_max=7, xi_pdfb=0.0, res_factor=1.0, t_max=1, xi_reweight=0.0)[0]
    assert rep["cycles"] == 1 and rep["iterations"] == 7
    it2 = _iterate(ctx, prob, prob.y)
    ctx.fhs_measure(0, it2[0]["X"], u0)            # u_prev = Phi X^(0)
    it2[0]["state"]["u_prev"].copy_(u0)
    ctx.fhs_pdfb_iter(it2, 7, want_stats=False)
    assert torch.equal(it1[0]["X"], it2[0]["X"])
    ctx.close()


def test_sara_limit_keeps_nuclear_duals_zero():
    """C = L and mu_bar = 0 (Section 2.4.1): Faceted HyperSARA reduces to per-channel SARA;
    the nuclear duals stay zero and X follows the oracle."""
    spec, inp, prob = make_problem("faceted", n=64, L=3, Q=2, m_ratio=0.5, B=1)
    prob.mu_bar = np.zeros_like(prob.mu_bar)
    ctx = make_context(prob, torch)
    it = _iterate(ctx, prob, prob.y)
    ctx.fhs_pdfb_iter(it, 6)
    assert float(it[0]["state"]["P"].abs().max()) == 0.0
    st = pd.initial_state(prob)
    for _ in range(6):
        pd.pdfb_iteration(prob, st)
    assert rel_err(it[0]["X"].double().cpu().numpy(), st.X) < 1e-4
    ctx.close()


def test_solve_reports_nonfinite_data(tiny):
    from paper_2003_07358_gb300.fhs import FhsError
    spec, inp, prob = tiny
    ctx = make_context(prob, torch)
    y = prob.y.copy()
    y[17] = complex(np.nan, 0.0)
    it = _iterate(ctx, prob, y)
    with pytest.raises(FhsError, match="NONFINITE"):
        ctx.fhs_solve(it, **RULES)
    # the context stays usable
    it2 = _iterate(ctx, prob, prob.y)
    rep = ctx.fhs_solve(it2, p_min=2, p_max=2, xi_pdfb=0.0, res_factor=1.0, t_max=1, xi_reweight=0.0)[0]
    assert rep["iterations"] == 2 and not rep["nonfinite"]
    ctx.close()


def test_host_buffer_iterations_match_device_ones(tiny):
    """fhs_pdfb_iter_host (data and result in host memory, caller's order) gives the
    iterates of fhs_pdfb_iter on the same data, bit for bit."""
    spec, inp, prob = tiny
    ctx = make_context(prob, torch)
    it1 = _iterate(ctx, prob, prob.y)
    s1 = ctx.fhs_pdfb_iter(it1, 5)
    X = torch.zeros((prob.L, prob.n1, prob.n2), device="cuda")
    it2 = [{"X": X, "Xcheck": torch.zeros_like(X), "y": torch.empty_like(it1[0]["y"]), "state": ctx.new_state(0)}]
    y_host = torch.as_tensor(np.ascontiguousarray(prob.y, dtype=np.complex64)).pin_memory()
    X_host = torch.empty((prob.L, prob.n1, prob.n2), dtype=torch.float32).pin_memory()
    s2 = ctx.fhs_pdfb_iter_host(it2, [y_host], [X_host], 5)
    assert torch.equal(X_host, it1[0]["X"].cpu())
    assert s1[0]["xi"] == s2[0]["xi"]
    ctx.close()
