"""Degenerate inputs through the C ABI against the FP64 oracle: a channel without
visibilities and an empty data block in the same cube (measure, adjoint and five PDFB
iterations of Algorithm 2), and the zero image with zero data, a fixed point of the
iteration (every dual and the primal stay exactly zero)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import nufft as nu
from oracle import pdfb as pd
from tests._fixtures import REL_TOL, make_context, make_problem, rel_err, to_dev_f32, vis_to_internal, vis_to_user

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _edge_problem():
    """tiny workload with L = 3, B = 2; channel 0 keeps only block 0, channel 1 loses
    every visibility, channel 2 is unchanged (step sizes and radii of the full problem)."""
    spec, inp, prob = make_problem("tiny", L=3, B=2)
    keep, M = [], np.zeros_like(prob.M_lb)
    for l, b, s in prob.vis_slices():
        if (l == 0 and b == 1) or l == 1:
            continue
        keep.append(np.arange(s.start, s.stop))
        M[l, b] = s.stop - s.start
    idx = np.concatenate(keep)
    prob.uv = np.ascontiguousarray(prob.uv[idx])
    prob.y = prob.y[idx]
    prob.M_lb = M
    return inp, prob


def test_empty_channel_and_block_operators():
    inp, prob = _edge_problem()
    ctx = make_context(prob, torch)
    x = inp.x_true
    y = torch.empty(prob.uv.shape[0], dtype=torch.complex64, device="cuda")
    ctx.fhs_measure(0, to_dev_f32(torch, x), y)
    got = vis_to_user(ctx, torch, y)
    ref = nu.measure_cube(x, prob.uv, prob.M_lb.sum(axis=1))
    assert rel_err(got, ref) < REL_TOL
    rng = np.random.default_rng(11)
    v = (rng.standard_normal(prob.uv.shape[0]) + 1j * rng.standard_normal(prob.uv.shape[0]))
    v = v.astype(np.complex64).astype(np.complex128)
    xa = torch.empty((prob.L, prob.n1, prob.n2), device="cuda")
    ctx.fhs_adjoint(0, vis_to_internal(ctx, torch, v), xa)
    ref = nu.adjoint_cube_real(v, prob.uv, prob.M_lb.sum(axis=1), prob.n1, prob.n2)
    got = xa.cpu().numpy()
    assert rel_err(got, ref) < REL_TOL
    assert np.all(got[1] == 0.0)                  # no visibilities: Phi_1^dagger = 0
    ctx.close()


def test_empty_channel_and_block_pdfb():
    inp, prob = _edge_problem()
    ctx = make_context(prob, torch)
    L, n1, n2 = prob.L, prob.n1, prob.n2
    X = torch.zeros((L, n1, n2), device="cuda")
    Xc = torch.zeros_like(X)
    st = ctx.new_state(0)
    it = [{"X": X, "Xcheck": Xc, "y": vis_to_internal(ctx, torch, prob.y), "state": st}]
    ctx.fhs_pdfb_iter(it, 5)
    ost = pd.initial_state(prob)
    for _ in range(5):
        pd.pdfb_iteration(prob, ost)
    assert rel_err(X.cpu().numpy(), ost.X) < 1e-4
    ctx.close()


def test_zero_image_is_a_fixed_point():
    spec, inp, prob = make_problem("faceted", L=4)
    ctx = make_context(prob, torch)
    X = torch.zeros((prob.L, prob.n1, prob.n2), device="cuda")
    Xc = torch.zeros_like(X)
    st = ctx.new_state(0)
    y0 = torch.zeros(prob.uv.shape[0], dtype=torch.complex64, device="cuda")
    it = [{"X": X, "Xcheck": Xc, "y": y0, "state": st}]
    stats = ctx.fhs_pdfb_iter(it, 3)
    assert torch.count_nonzero(X).item() == 0 and torch.count_nonzero(Xc).item() == 0
    assert torch.count_nonzero(st["W"]).item() == 0 and torch.count_nonzero(st["P"]).item() == 0
    assert torch.count_nonzero(st["v"]).item() == 0
    assert stats[0]["res_norm"] == 0.0
    ctx.close()
