"""Checkpoints and the error paths, exercised without faulting the GPU:

* fhs_checkpoint_save / _load: the iterations resume bit for bit; a corrupt file or a
  context of another shape is refused before anything changes;
* a bounded device-side wait that runs out (first phase shortened by the test hook, the
  drain phase at full length so every copy and MMA lands) is reported as TIMEOUT by the
  next synchronising call, and later calls work;
* an allocation cap makes fhs_create fail with OOM;
* NaN data makes the iteration statistics report NONFINITE.
"""
from __future__ import annotations

import numpy as np
import pytest

from _fixtures import make_context, make_problem, vis_to_internal

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tiny():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return make_problem("tiny")


def _iterate(ctx, prob, y_user=None):
    X = torch.zeros((prob.L, prob.n1, prob.n2), device="cuda")
    return [{"X": X, "Xcheck": torch.zeros_like(X),
             "y": vis_to_internal(ctx, torch, prob.y if y_user is None else y_user), "state": ctx.new_state(0)}]


def test_checkpoint_resumes_bit_for_bit(tiny, tmp_path):
    from paper_2003_07358_gb300.fhs import FhsError
    spec, inp, prob = tiny
    ctx = make_context(prob, torch)
    a = _iterate(ctx, prob)
    ctx.fhs_pdfb_iter(a, 5, want_stats=False)
    ctx.fhs_reweight(0, a[0]["X"], a[0]["state"]["theta"], a[0]["state"]["theta_bar"])
    path = str(tmp_path / "state.ckpt")
    ctx.fhs_checkpoint_save(a, path)
    ctx.fhs_pdfb_iter(a, 5, want_stats=False)
    b = _iterate(ctx, prob)
    ctx.fhs_checkpoint_load(b, path)
    ctx.fhs_pdfb_iter(b, 5, want_stats=False)
    for key in ("X", "Xcheck"):
        assert torch.equal(a[0][key], b[0][key])
    for key in ("W", "P", "v", "u_prev", "theta", "theta_bar"):
        assert torch.equal(a[0]["state"][key], b[0]["state"][key]), key
    # a corrupt file is refused and leaves the arrays untouched
    raw = bytearray(open(path, "rb").read())
    raw[len(raw) // 2] ^= 0x40
    bad = str(tmp_path / "bad.ckpt")
    open(bad, "wb").write(bytes(raw))
    before = b[0]["X"].clone()
    with pytest.raises(FhsError, match="corrupt"):
        ctx.fhs_checkpoint_load(b, bad)
    assert torch.equal(before, b[0]["X"])
    ctx.close()
    # a context of another shape is refused
    spec2, inp2, prob2 = make_problem("tiny", n=32, L=4, m_abs=300)
    ctx2 = make_context(prob2, torch)
    with pytest.raises(FhsError, match="shape"):
        ctx2.fhs_checkpoint_load(_iterate(ctx2, prob2), path)
    ctx2.close()


def test_wait_timeout_is_reported_and_recovered(tiny):
    from paper_2003_07358_gb300.fhs import FhsError, fhs_set_wait_limit
    spec, inp, prob = tiny
    ctx = make_context(prob, torch)
    ref = _iterate(ctx, prob)
    ctx.fhs_pdfb_iter(ref, 3, want_stats=False)
    ctx.sync()
    a = _iterate(ctx, prob)
    try:
        fhs_set_wait_limit(-1)                     # every first phase gives up at once
        ctx.fhs_pdfb_iter(a, 1, want_stats=False)
        with pytest.raises(FhsError, match="TIMEOUT"):
            ctx.sync()
    finally:
        fhs_set_wait_limit(0)
    ctx.sync()                                     # the status word was cleared
    b = _iterate(ctx, prob)
    ctx.fhs_pdfb_iter(b, 3, want_stats=False)
    ctx.sync()
    assert torch.equal(b[0]["X"], ref[0]["X"])
    ctx.close()


def test_allocation_cap_gives_oom(tiny):
    from paper_2003_07358_gb300.fhs import FhsError, fhs_set_alloc_limit
    spec, inp, prob = tiny
    try:
        fhs_set_alloc_limit(1 << 16)
        with pytest.raises(FhsError, match="OOM"):
            make_context(prob, torch)
    finally:
        fhs_set_alloc_limit(0)
    ctx = make_context(prob, torch)
    ctx.close()


def test_nan_data_reported_as_nonfinite(tiny):
    from paper_2003_07358_gb300.fhs import FhsError
    spec, inp, prob = tiny
    ctx = make_context(prob, torch)
    y = prob.y.copy()
    y[3] = complex(np.nan, 0.0)
    a = _iterate(ctx, prob, y)
    with pytest.raises(FhsError, match="NONFINITE"):
        ctx.fhs_pdfb_iter(a, 2)
    b = _iterate(ctx, prob)
    assert np.isfinite(ctx.fhs_pdfb_iter(b, 2)[0]["xi"])
    ctx.close()
