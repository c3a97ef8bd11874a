"""Batching form: several independent cubes of uneven sizes (image side, channels,
facets, visibility density, blocks), each with its own seed, held by one context and
iterated together by fhs_pdfb_iter (one CUDA graph over all cubes).  Every cube must
match its own FP64 oracle run (Algorithm 2 per sub-cube, Section 2.4.1: sub-cubes are
independent problems)."""
from __future__ import annotations

import numpy as np
import pytest

import fhs_synth as fs
from oracle import pdfb as pd

from _fixtures import rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# (n, L, Q, M/N, B, window, seed): sizes span the batch's ranges at test scale
CUBES = [
    (32, 3, 1, 0.3, 1, "triangular", 31),
    (64, 5, 2, 2.0, 2, "sine", 32),
    (128, 2, 3, 0.5, 1, "triangular", 33),
    (64, 8, 1, 1.0, 3, "triangular", 34),
    (32, 6, 2, 1.5, 2, "sine", 35),
]


def _problem(n, L, Q, mr, B, window, seed):
    spec = fs.CubeSpec(f"batch cube n={n} L={L} Q={Q}", n=n, L=L, C=1, Q=Q, overlap=0.1, window=window,
                       m_ratio=mr, B=B, isnr_db=40.0, n_blobs=8, seed=seed)
    inp = fs.make_inputs(spec)
    prob, _ = pd.build_problem(inp, power_iters=30)
    prob.y = prob.y.astype(np.complex64).astype(np.complex128)
    return prob


@pytest.fixture(scope="module")
def batch():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2003_07358_gb300.fhs import Context, CubeParams
    probs = [_problem(*c) for c in CUBES]
    cps = [CubeParams(n1=p.n1, n2=p.n2, L=p.L, Qy=p.Qy, Qx=p.Qx, overlap=p.rho, window=p.window, M_lb=p.M_lb,
                      uv=p.uv, eta=p.eta, mu=p.mu, mu_bar=p.mu_bar, eps=p.eps, tau=p.tau, zeta=p.zeta,
                      kappa=p.kappa) for p in probs]
    ctx = Context(cps)
    yield probs, ctx
    ctx.close()


def test_batch_of_uneven_cubes_matches_oracle_per_cube(batch):
    probs, ctx = batch
    its = []
    for c, p in enumerate(probs):
        X = torch.zeros((p.L, p.n1, p.n2), device="cuda")
        u = torch.as_tensor(np.ascontiguousarray(p.y, dtype=np.complex64), device="cuda")
        y = torch.empty_like(u)
        ctx.fhs_vis_to_internal(c, u, y)
        its.append({"X": X, "Xcheck": torch.zeros_like(X), "y": y, "state": ctx.new_state(c)})
    n_iter = 4
    stats = ctx.fhs_pdfb_iter(its, n_iter)
    for c, p in enumerate(probs):
        st = pd.initial_state(p)
        for _ in range(n_iter):
            out = pd.pdfb_iteration(p, st)
        err = rel_err(its[c]["X"].cpu().numpy(), st.X)
        assert err < 1e-4, (c, err)
        assert stats[c]["xi"] == pytest.approx(out["xi"], rel=1e-3)


def test_batch_graph_replays_match_single_cube_contexts(batch):
    """The batched context and one context per cube give the same iterates."""
    probs, ctx = batch
    from paper_2003_07358_gb300.fhs import Context, CubeParams
    its = []
    for c, p in enumerate(probs):
        X = torch.zeros((p.L, p.n1, p.n2), device="cuda")
        u = torch.as_tensor(np.ascontiguousarray(p.y, dtype=np.complex64), device="cuda")
        y = torch.empty_like(u)
        ctx.fhs_vis_to_internal(c, u, y)
        its.append({"X": X, "Xcheck": torch.zeros_like(X), "y": y, "state": ctx.new_state(c)})
    ctx.fhs_pdfb_iter(its, 3, want_stats=False)
    for c in (1, 3):
        p = probs[c]
        one = Context([CubeParams(n1=p.n1, n2=p.n2, L=p.L, Qy=p.Qy, Qx=p.Qx, overlap=p.rho, window=p.window,
                                  M_lb=p.M_lb, uv=p.uv, eta=p.eta, mu=p.mu, mu_bar=p.mu_bar, eps=p.eps, tau=p.tau,
                                  zeta=p.zeta, kappa=p.kappa)])
        X = torch.zeros((p.L, p.n1, p.n2), device="cuda")
        u = torch.as_tensor(np.ascontiguousarray(p.y, dtype=np.complex64), device="cuda")
        y = torch.empty_like(u)
        one.fhs_vis_to_internal(0, u, y)
        it1 = [{"X": X, "Xcheck": torch.zeros_like(X), "y": y, "state": one.new_state(0)}]
        one.fhs_pdfb_iter(it1, 3, want_stats=False)
        assert torch.equal(X, its[c]["X"]), c
        one.close()


@pytest.mark.parametrize("lanes", [2, 4])
def test_lanes_equal_one_lane_bit_for_bit(batch, lanes):
    """fhs_set_lanes: the cubes dealt to further lanes (own streams and scratch, run
    beside the first lane inside the iteration graph) give the same iterates, bit for
    bit, as one lane; the lane count is reported."""
    probs, ctx = batch

    def run(lanes):
        ctx.fhs_set_lanes(lanes)
        its = []
        for c, p in enumerate(probs):
            X = torch.zeros((p.L, p.n1, p.n2), device="cuda")
            u = torch.as_tensor(np.ascontiguousarray(p.y, dtype=np.complex64), device="cuda")
            y = torch.empty_like(u)
            ctx.fhs_vis_to_internal(c, u, y)
            its.append({"X": X, "Xcheck": torch.zeros_like(X), "y": y, "state": ctx.new_state(c)})
        stats = ctx.fhs_pdfb_iter(its, 3)
        return its, stats, ctx.fhs_get_lanes()

    two, st2, n2 = run(lanes)
    one, st1, n1 = run(1)
    assert (n2, n1) == (lanes, 1)
    for c in range(len(probs)):
        assert torch.equal(two[c]["X"], one[c]["X"]), c
        assert torch.equal(two[c]["state"]["W"], one[c]["state"]["W"]), c
        assert torch.equal(two[c]["state"]["v"], one[c]["state"]["v"]), c
        assert st2[c] == st1[c], c
    with pytest.raises(Exception):
        ctx.fhs_set_lanes(5)
