"""Shared set-up for the GPU parity tests: one seeded synthetic problem, the
FP64 oracle's Problem for it, and a libfhs Context built from the same inputs
(parameters computed once by the oracle and passed unchanged to both sides)."""
from __future__ import annotations

import numpy as np

import fhs_synth as fs
from oracle import pdfb as pd

REL_TOL = 1e-5          # per-operator relative error of the FP32 path against FP64


def rel_err(got, ref) -> float:
    got = np.asarray(got, dtype=np.complex128 if np.iscomplexobj(got) or np.iscomplexobj(ref) else np.float64)
    ref = np.asarray(ref)
    return float(np.linalg.norm((got - ref).ravel()) / max(np.linalg.norm(np.ravel(ref)), 1e-300))


def make_problem(name: str, power_iters: int = 30, **over):
    spec = fs.workload(name, **over)
    inp = fs.make_inputs(spec)
    prob, aux = pd.build_problem(inp, power_iters=power_iters)
    # both sides see the complex64 data the GPU holds
    prob.y = prob.y.astype(np.complex64).astype(np.complex128)
    return spec, inp, prob


def make_context(prob, torch):
    from paper_2003_07358_gb300.fhs import Context, CubeParams
    cp = CubeParams(n1=prob.n1, n2=prob.n2, L=prob.L, Qy=prob.Qy, Qx=prob.Qx, overlap=prob.rho,
                    window=prob.window, M_lb=prob.M_lb, uv=prob.uv, eta=prob.eta, mu=prob.mu,
                    mu_bar=prob.mu_bar, eps=prob.eps, tau=prob.tau, zeta=prob.zeta, kappa=prob.kappa)
    return Context([cp])


def to_dev_c64(torch, a, device="cuda"):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.complex64), device=device)


def to_dev_f32(torch, a, device="cuda"):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=device)


def vis_to_internal(ctx, torch, user_c128):
    u = to_dev_c64(torch, user_c128)
    out = torch.empty_like(u)
    ctx.fhs_vis_to_internal(0, u, out)
    return out


def vis_to_user(ctx, torch, internal):
    out = torch.empty_like(internal)
    ctx.fhs_vis_to_user(0, internal, out)
    return out.cpu().numpy().astype(np.complex128)
