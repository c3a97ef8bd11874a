"""The allocation-free l2-ball projection (for callers that may not allocate
device memory, so cannot create a context) gives the same result as the
context-based fhs_proj_l2ball_blocks, on two calls in a row through the C ABI.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
import numpy as np
import pytest

from tests._fixtures import REL_TOL, make_context, make_problem, rel_err, vis_to_internal, vis_to_user

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _segments(prob):
    """(l, b) blocks of the caller's order as contiguous segments."""
    off = [0]
    eps = []
    for (l, b, sl) in prob.vis_slices():
        off.append(sl.stop)
        eps.append(prob.eps[l, b])
    return np.array(off, dtype=np.int64), np.array(eps)


def test_noalloc_matches_context_projection_twice():
    from paper_2003_07358_gb300.fhs import fhs_proj_l2ball_noalloc
    spec, inp, prob = make_problem("faceted", n=128, L=3, Q=2, m_ratio=0.37, B=3)
    ctx = make_context(prob, torch)
    seg_off, eps = _segments(prob)
    rng = np.random.default_rng(21)
    M = prob.uv.shape[0]
    for call in range(2):
        z = prob.y + (0.3 + call) * (rng.standard_normal(M) + 1j * rng.standard_normal(M)) * np.abs(prob.y).mean()
        if call == 1:   # one segment inside its ball on the second call
            l0, b0, s0 = prob.vis_slices()[2]
            z[s0] = prob.y[s0] + (z[s0] - prob.y[s0]) * (0.5 * eps[2] / np.linalg.norm(z[s0] - prob.y[s0]))
        z = z.astype(np.complex64)
        # existing entry point (context, internal order)
        zi, yi = vis_to_internal(ctx, torch, z), vis_to_internal(ctx, torch, prob.y)
        vi = torch.empty_like(zi)
        dn_ref = ctx.fhs_proj_l2ball_blocks(0, zi, yi, vi)
        ref = vis_to_user(ctx, torch, vi)
        # allocation-free entry point (plain arrays, caller's order)
        zd = torch.as_tensor(z, device="cuda")
        yd = torch.as_tensor(prob.y.astype(np.complex64), device="cuda")
        vd = torch.full_like(zd, complex(np.nan, np.nan))
        dn = fhs_proj_l2ball_noalloc(zd, yd, seg_off, eps, vd)
        got = vd.cpu().numpy().astype(np.complex128)
        assert np.all(np.isfinite(got))
        assert rel_err(got, ref) < REL_TOL
        assert np.max(np.abs(got - ref)) <= REL_TOL * np.max(np.abs(ref))
        # the context path squares the float-rounded z - y, this one the exact difference
        assert np.allclose(dn, dn_ref, rtol=REL_TOL)
        if call == 1:
            assert np.all(got[s0] == 0)
    ctx.close()


def test_noalloc_rejects_too_many_segments():
    from paper_2003_07358_gb300.fhs import FhsError, fhs_proj_l2ball_noalloc
    z = torch.zeros(100, dtype=torch.complex64, device="cuda")
    v = torch.empty_like(z)
    off = np.linspace(0, 100, 66).astype(np.int64)      # 65 segments > 64
    with pytest.raises(FhsError, match="nseg"):
        fhs_proj_l2ball_noalloc(z, z, off, np.ones(65), v)


def test_noalloc_nonfinite_input_is_never_a_silent_zero():
    """A NaN in z makes its segment's v NaN when the norms are not requested (the call
    does not synchronise), and the call reports NONFINITE when they are."""
    from paper_2003_07358_gb300.fhs import FhsError, fhs_proj_l2ball_noalloc
    rng = np.random.default_rng(5)
    z = torch.as_tensor((rng.standard_normal(300) + 1j * rng.standard_normal(300)).astype(np.complex64), device="cuda")
    y = torch.zeros_like(z)
    z[150] = complex(float("nan"), 0.0)
    off = np.array([0, 100, 300], dtype=np.int64)
    v = torch.empty_like(z)
    fhs_proj_l2ball_noalloc(z, y, off, np.array([1.0, 1.0]), v, want_norms=False)
    got = v.cpu().numpy()
    assert np.all(np.isnan(got[100:300]))
    assert np.all(np.isfinite(got[:100]))
    with pytest.raises(FhsError, match="NONFINITE"):
        fhs_proj_l2ball_noalloc(z, y, off, np.array([1.0, 1.0]), v)
