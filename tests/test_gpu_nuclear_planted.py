"""Nuclear dual (Table 2 row 2, Algorithm 2 P update) on a facet with planted singular
values spread over five decades and thresholds between them, so that the result depends
on the small singular values: P = U diag(min(s, alpha)) V^T in closed form.  Checked on
the fast path (error-free Gram on tcgen05 tensor cores) and on the plain path
(float-float Gram on CUDA cores), for 16 and 32 channels.  A Gram accumulated in FP32
(errors ~2^-24 s_max^2) would miss the components whose s_j^2 is below that."""
from __future__ import annotations

import numpy as np
import pytest

from _fixtures import rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _context(n, L):
    from paper_2003_07358_gb300.fhs import Context, CubeParams
    rng = np.random.default_rng(1)
    M_lb = np.full((L, 1), 64, dtype=np.int64)
    uv = rng.uniform(-1.0, 1.0, (64 * L, 2)).astype(np.float32)
    cp = CubeParams(n1=n, n2=n, L=L, Qy=1, Qx=1, overlap=0.1, window="triangular", M_lb=M_lb, uv=uv,
                    eta=np.ones(L), mu=0.1, mu_bar=np.ones(1), eps=np.ones((L, 1)))
    return Context([cp])


@pytest.mark.parametrize("L", [16, 32])
@pytest.mark.parametrize("path", ["fast", "plain"])
def test_nuclear_dual_planted_wide_spectrum(L, path):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    n = 128
    N = n * n
    rng = np.random.default_rng(L)
    U, _ = np.linalg.qr(rng.standard_normal((N, L)))
    V, _ = np.linalg.qr(rng.standard_normal((L, L)))
    s = 10.0 * np.logspace(0, -5, L)                    # 10 .. 1e-4
    Z = (U * s) @ V.T                                   # [pixels][channels]
    Z = Z.astype(np.float32).astype(np.float64)         # the GPU holds FP32 images
    U2, s2, Vt2 = np.linalg.svd(Z, full_matrices=False)  # exact SVD of the FP32 matrix
    # thresholds between consecutive singular values: every component is in play
    alpha = np.sqrt(s2 * np.concatenate([s2[1:], s2[-1:] * 0.1]))
    tb = (alpha / alpha.max()).astype(np.float32)       # theta_bar in ]0, 1], mu_bar = max alpha
    mu_bar = float(alpha.max())
    alpha = mu_bar * tb.astype(np.float64)
    ref = (U2 * np.minimum(s2, alpha)) @ Vt2
    ctx = _context(n, L)
    ctx.fhs_set_params(0, 0.33, 1.0, 1.0, np.ones(L), 0.1, np.array([mu_bar]), np.ones(L))
    ctx.fhs_set_path(path)
    X = torch.as_tensor(np.ascontiguousarray(Z.T.reshape(L, n, n), dtype=np.float32), device="cuda")
    P = torch.zeros(L * N, device="cuda")
    A = torch.zeros((L, n, n), device="cuda")
    ctx.fhs_prox_nuclear_facets(0, X, P, torch.as_tensor(tb[None, :], device="cuda"), A)
    got = P.double().cpu().numpy().reshape(L, N).T
    assert rel_err(got, ref) < 1e-5
    # the smallest component (s ~ 1e-4 of s_max) is resolved: its coefficient matches
    c = (U2[:, -1] @ got @ Vt2[-1])
    assert c == pytest.approx(min(s2[-1], alpha[-1]), rel=1e-2)
    ctx.close()
