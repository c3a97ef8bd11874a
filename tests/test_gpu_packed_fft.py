"""Parity of the measurement operator and its adjoint at grid sizes 2048 and 4096
(1024^2 and 2048^2 images), where the fast path transforms two image columns per
complex column: the forward recovers both real columns' transforms from Hermitian
symmetry in the row DFT, the adjoint packs the Hermitian parts of two columns so that
one complex column DFT yields both real outputs.  Phi x and Re Phi^dagger v over every
visibility and pixel of two channels against the FP64 oracle (Eq. 1), and the adjoint
pairing."""
from __future__ import annotations

import numpy as np
import pytest

import fhs_synth as fs
from oracle import nufft as nu

from _fixtures import REL_TOL, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[1024, 2048])
def mid(request):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2003_07358_gb300.fhs import Context, CubeParams
    n = request.param
    spec = fs.workload("tiny", n=n, L=2, m_abs=40000, Q=1)
    inp = fs.make_inputs(spec, with_noise=False)
    L = spec.L
    M_lb = inp.M_lb
    uv = inp.uv
    cp = CubeParams(n1=n, n2=n, L=L, Qy=1, Qx=1, overlap=0.1, window="triangular", M_lb=M_lb, uv=uv,
                    eta=np.ones(L), mu=0.0, mu_bar=np.zeros(1), eps=np.ones((L, 1)))
    ctx = Context([cp])
    x = inp.x_true.astype(np.float32)
    xd = torch.as_tensor(x, device="cuda")
    y = torch.empty(uv.shape[0], dtype=torch.complex64, device="cuda")
    ctx.fhs_measure(0, xd, y)
    yu = torch.empty_like(y)
    ctx.fhs_vis_to_user(0, y, yu)
    ctx.sync()
    yield dict(torch=torch, ctx=ctx, x=x, xd=xd, y=y, yu=yu, uv=uv, M_l=M_lb.sum(axis=1), n=n)
    ctx.close()


def test_measure_packed_matches_oracle(mid):
    ref = nu.measure_cube(mid["x"].astype(np.float64), mid["uv"], mid["M_l"])
    got = mid["yu"].cpu().numpy().astype(np.complex128)
    assert rel_err(got, ref) < REL_TOL
    assert np.abs(got - ref).max() <= 4 * REL_TOL * np.abs(ref).max()


def test_adjoint_pairing_packed(mid):
    torch = mid["torch"]
    out = torch.empty_like(mid["xd"])
    mid["ctx"].fhs_adjoint(0, mid["y"], out)
    mid["ctx"].sync()
    a = float((mid["y"].abs().double() ** 2).sum())
    b = float((mid["xd"].double() * out.double()).sum())
    assert abs(a - b) <= REL_TOL * a, (a, b)


def test_adjoint_packed_matches_oracle(mid):
    """Re Phi^dagger v over the whole cube against the FP64 oracle (Algorithm 2 adjoint)."""
    torch = mid["torch"]
    rng = np.random.default_rng(7)
    nv = mid["uv"].shape[0]
    v = (rng.standard_normal(nv) + 1j * rng.standard_normal(nv)).astype(np.complex64)
    vu = torch.as_tensor(v, device="cuda")
    vi = torch.empty_like(vu)
    mid["ctx"].fhs_vis_to_internal(0, vu, vi)
    out = torch.empty_like(mid["xd"])
    mid["ctx"].fhs_adjoint(0, vi, out)
    got = out.cpu().numpy().astype(np.float64)
    ref = nu.adjoint_cube_real(v.astype(np.complex128), mid["uv"], mid["M_l"], mid["n"], mid["n"])
    assert rel_err(got, ref) < REL_TOL
    assert np.abs(got - ref).max() <= 4 * REL_TOL * np.abs(ref).max()
