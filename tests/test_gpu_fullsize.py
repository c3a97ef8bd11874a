"""Parity at the full bench size: one 4096 x 4096 x 16 sub-cube with 8,388,608
visibilities per channel (K = 8192 grid, 16 x 16 facets), the launch configuration
bench.py times.  The FP64 oracle cannot run the whole operator there, so it is
compared on sampled outputs it computes one by one (Eq. 1 at chosen visibilities
and pixels); the adjoint pairing holds at any size and is checked in full."""
from __future__ import annotations

import numpy as np
import pytest

import fhs_synth as fs
from oracle import nufft as nu

from _fixtures import REL_TOL, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2003_07358_gb300.fhs import Context, CubeParams
    spec = fs.workload("large")
    rng = np.random.default_rng(spec.seed)
    sources = fs.sky_sources(spec, rng)
    base = fs.base_uv(spec, rng)
    blocks = fs.radial_blocks(base, spec.B)
    perm = np.concatenate(blocks)
    chans = fs.subcube_channels(spec, 0)
    Lc, n = spec.Lc, spec.n
    M_lb = np.array([[b.size for b in blocks]] * Lc, dtype=np.int64)
    uv = np.concatenate([fs.channel_uv(base, spec, l)[perm] for l in chans])
    cp = CubeParams(n1=n, n2=n, L=Lc, Qy=spec.Q, Qx=spec.Q, overlap=spec.overlap, window=spec.window, M_lb=M_lb,
                    uv=uv, eta=np.ones(Lc), mu=0.0, mu_bar=np.zeros(spec.Q * spec.Q), eps=np.ones((Lc, spec.B)))
    ctx = Context([cp])
    x = np.stack([fs.render_channel(spec, sources, int(l)).astype(np.float32) for l in chans])
    xd = torch.as_tensor(x, device="cuda")
    nv = int(M_lb.sum())
    y = torch.empty(nv, dtype=torch.complex64, device="cuda")
    ctx.fhs_measure(0, xd, y)
    yu = torch.empty_like(y)
    ctx.fhs_vis_to_user(0, y, yu)
    ctx.sync()
    Ml = int(M_lb[0].sum())
    yield dict(torch=torch, ctx=ctx, x=x, xd=xd, y=y, yu=yu, uv=uv, Ml=Ml, n=n, Lc=Lc)
    del ctx
    torch.cuda.empty_cache()


def test_measure_fullsize_sampled(big):
    """Phi x at 3 channels x 24 random visibilities against the FFT-free oracle evaluation."""
    rng = np.random.default_rng(5)
    got, want = [], []
    for l in (0, 7, big["Lc"] - 1):
        idx = np.sort(rng.choice(big["Ml"], size=24, replace=False)) + l * big["Ml"]
        got.append(big["yu"][big["torch"].as_tensor(idx, device="cuda")].cpu().numpy())
        want.append(nu.measure_sampled(big["x"][l].astype(np.float64), big["uv"][idx]))
    err = rel_err(np.concatenate(got), np.concatenate(want))
    assert err <= REL_TOL, err


def test_adjoint_pairing_fullsize(big):
    """<Phi x, Phi x> = <x, Re Phi^dagger Phi x> over the whole sub-cube (holds at any size)."""
    torch = big["torch"]
    out = torch.empty_like(big["xd"])
    big["ctx"].fhs_adjoint(0, big["y"], out)
    big["ctx"].sync()
    a = float((big["y"].abs().double() ** 2).sum())
    b = float((big["xd"].double() * out.double()).sum())
    assert abs(a - b) <= REL_TOL * a, (a, b)


def test_adjoint_fullsize_sampled_pixels(big):
    """Re Phi^dagger y of channel 0 at five pixels by direct summation over its 8.4M
    visibilities; error bounded by REL_TOL of the image's largest magnitude."""
    torch = big["torch"]
    out = torch.empty_like(big["xd"])
    big["ctx"].fhs_adjoint(0, big["y"], out)
    img = out[0].cpu().numpy().astype(np.float64)
    n, Ml = big["n"], big["Ml"]
    r0, c0 = np.unravel_index(np.argmax(big["x"][0]), big["x"][0].shape)
    pix = [(int(r0), int(c0)), (n // 2, n // 2), (0, 0), (n - 1, 17), (1234, 3071)]
    v = big["yu"][:Ml].cpu().numpy().astype(np.complex128)
    want = nu.adjoint_real_sampled(v, big["uv"][:Ml], n, n, pix)
    got = np.array([img[r, c] for r, c in pix])
    assert np.abs(got - want).max() <= REL_TOL * np.abs(img).max(), (got, want)
