#!/usr/bin/env python
"""PDFB iterations per second of the Faceted HyperSARA hot path on GB300.

Workload (default "large"): 4096 x 4096 image, 64 channels as 4 channel-
interleaved sub-cubes of 16, 16 x 16 spatial facets (10 % nuclear overlap),
M = 0.5 N = 8,388,608 visibilities per channel in 8 uv-radial blocks, iSNR
30 dB; synthetic sky (Gaussian blobs + point sources with curved power-law
spectra) and Gaussian uv coverage scaled with frequency.  One step = one
iteration of Algorithm 2 on all 4 sub-cubes.  Inputs are resident in HBM
(working set ~100 GB, far above the 129 MB L2, so no flush is needed).

--impl reference times the FP64 oracle (test infrastructure) on the host
cores on a bounded sample of the same workload, scaled to one iteration.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import fhs_synth as fs  # noqa: E402

METRIC = "PDFB iter/s at 4096^2 x 64ch"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="large", choices=list(fs.WORKLOADS))
    ap.add_argument("--opnorm-iters", type=int, default=20)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ops", action="store_true")
    ap.add_argument("--plain-steps", type=int, default=2)
    ap.add_argument("--no-snr-gap", action="store_true")
    ap.add_argument("--no-dde", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--lanes", type=int, default=1, choices=[1, 2, 3, 4],
                    help="fhs_set_lanes: sub-cubes of an iteration on 1 to 4 concurrent lanes")
    ap.add_argument("--autotune", type=int, default=0, choices=[0, 1, 2],
                    help="fhs_set_autotune mode for the contexts of the bench (0 defaults, 1 cache then measure, "
                         "2 measure); the choices are reported per shape")
    ap.add_argument("--dry-run", action="store_true",
                    help="set up the ranks (gloo, CPU) and print each rank's sub-cube seed offset, nothing else")
    return ap.parse_args()


def relaunch_under_torchrun(args) -> int:
    """--gpus N > 1 without a launcher: start N ranks with torch.distributed.run (one
    independent replica of the workload per rank, no data-path collective)."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def dry_run(args):
    """Rank set-up only (CPU, gloo): each rank reports the seed offset of its replica."""
    from paper_2003_07358_gb300 import sharding as sh
    info = sh.rank_info()
    if info.world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        dist.barrier()
    line = json.dumps({"dry_run": True, "rank": info.rank, "world": info.world, "seed_offset": info.rank,
                       "workload": fs.WORKLOADS[args.workload].name})
    os.write(1, (line + "\n").encode())      # one write: lines of concurrent ranks do not interleave
    if info.world > 1:
        dist.destroy_process_group()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.flush()
        rows = []
        with open(self.out.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.out.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# -------------------------------------------------------------- workload
def chi_mean_std(k: int):
    m = math.sqrt(2.0) * math.exp(math.lgamma((k + 1) / 2.0) - math.lgamma(k / 2.0))
    return m, math.sqrt(max(k - m * m, 0.0))


def facet_pixels(n: int, Q: int, rho: float) -> list[int]:
    tb = [(i * n) // Q for i in range(Q + 1)]
    side = [(tb[i + 1] - tb[i]) + (0 if i == 0 else int(math.floor(rho * (tb[i + 1] - tb[i])))) for i in range(Q)]
    return [a * b for a in side for b in side]


def setup(spec: fs.CubeSpec, torch, seed_offset: int, opnorm_iters: int, log):
    """Create the context, the data y = Phi x + noise, the parameters and the state of every sub-cube."""
    from paper_2003_07358_gb300.fhs import Context, CubeParams
    rng = np.random.default_rng(spec.seed + seed_offset)
    sources = fs.sky_sources(spec, rng)
    base = fs.base_uv(spec, rng)
    blocks = fs.radial_blocks(base, spec.B)
    perm = np.concatenate(blocks)
    Lc, n, Q = spec.Lc, spec.n, spec.Q
    M_lb = np.array([[b.size for b in blocks]] * Lc, dtype=np.int64)
    cubes = []
    t0 = time.time()
    for c in range(spec.C):
        chans = fs.subcube_channels(spec, c)
        uv = np.concatenate([fs.channel_uv(base, spec, l)[perm] for l in chans])
        cubes.append(CubeParams(n1=n, n2=n, L=Lc, Qy=Q, Qx=Q, overlap=spec.overlap, window=spec.window, M_lb=M_lb,
                                uv=uv, eta=np.ones(Lc), mu=0.0, mu_bar=np.zeros(Q * Q), eps=np.zeros((Lc, spec.B))))
    ctx = Context(cubes)
    del cubes
    log(f"context created in {time.time() - t0:.1f} s")
    dev = ctx.device
    iterates = []
    npix = facet_pixels(n, Q, spec.overlap)
    gen = torch.Generator(device=dev)
    for c in range(spec.C):
        chans = fs.subcube_channels(spec, c)
        sz = ctx.sizes(c)
        x = torch.empty((Lc, n, n), device=dev)
        for i, l in enumerate(chans):
            x[i].copy_(torch.from_numpy(fs.render_channel(spec, sources, int(l)).astype(np.float32)))
        y = torch.empty(sz["n_vis"], dtype=torch.complex64, device=dev)
        ctx.fhs_measure(c, x, y)
        del x
        zero = torch.zeros_like(y)
        tmp = torch.empty_like(y)
        dn = ctx.fhs_proj_l2ball_blocks(c, y, zero, tmp).reshape(Lc, spec.B)
        del zero, tmp
        Ml = M_lb.sum(axis=1)
        sigma = np.sqrt((dn ** 2).sum(axis=1)) / np.sqrt(Ml) * 10 ** (-spec.isnr_db / 20)
        gen.manual_seed(spec.seed * 100 + seed_offset * 10 + c)
        off = 0
        for i in range(Lc):
            m = int(Ml[i])
            noise = torch.randn(m, dtype=torch.complex64, device=dev, generator=gen)
            y[off:off + m] += float(sigma[i]) * noise
            off += m
        e2 = sigma ** 2 * (Ml + 2 * np.sqrt(Ml))
        eps = np.sqrt(e2[:, None] * M_lb / Ml[:, None])
        opn = ctx.fhs_opnorm_sq(c, opnorm_iters, 1e-4)
        sb = sigma / np.sqrt(opn)
        sbar = math.sqrt(float(np.mean(sb ** 2)))
        m_, s_ = chi_mean_std(Lc)
        mu = sbar * (m_ + s_)
        mu_bar = np.array([sbar * math.sqrt(p * Lc / min(p, Lc)) for p in npix])
        ctx.fhs_set_params(c, 0.33, 1.0, 1.0, 1.0 / opn, mu, mu_bar, eps)
        X = torch.zeros((Lc, n, n), device=dev)
        iterates.append({"X": X, "Xcheck": torch.zeros_like(X), "y": y, "state": ctx.new_state(c)})
    ctx.sync()
    log(f"data, parameters and state ready in {time.time() - t0:.1f} s")
    return ctx, iterates


# --------------------------------------------- DDE-extended de-gridding (Section 2.1)
DDE_WORKLOAD = "facet_slice"
DDE_S_A = 5            # 5 x 5 per antenna -> 9 x 9 per baseline -> 15 x 15 footprints
DDE_N_ANT = 27         # 351 baselines


def dde_flops_per_vis(S_d: int) -> int:
    """FP32 flops of one visibility in either direction (2 per FMA): column pass
    F S_d x 7 complex-by-real, row pass S_d^2 x 7, kernel product S_d^2 complex."""
    F = 7 + S_d - 1
    return 2 * (14 * F * S_d + 14 * S_d * S_d + 4 * S_d * S_d)


def dde_measurement(args, torch, log, sm_mhz) -> dict:
    """Both DDE kernels inside PDFB iterations of the 1024^2 x 16 workload with 15 x 15
    footprints, their ALU roofline (FP32 FMA pipe: 152 SMs x 128 lanes x 2 flops x
    clock), and the oracle's de-gridding + gridding on a sample of the same rows."""
    from oracle import dde as odde
    spec = fs.workload(DDE_WORKLOAD)
    ctx, its = setup(spec, torch, 0, 10, log)
    rng = np.random.default_rng(spec.seed)
    fs.sky_sources(spec, rng)
    base = fs.base_uv(spec, rng)
    perm = np.concatenate(fs.radial_blocks(base, spec.B))
    chans = fs.subcube_channels(spec, 0)
    shim = type("Inp", (), {"spec": spec, "chans": chans, "perm": perm})()
    dd = fs.dde_inputs(shim, n_ant=DDE_N_ANT, S_a=DDE_S_A)
    S_d = dd.kern.shape[1]
    stream = ctx.stream

    def timed_iters(k):
        ctx.fhs_pdfb_iter(its, 1, want_stats=False)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            ctx.fhs_pdfb_iter(its, 1, want_stats=False)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    plain_ms = timed_iters(3)
    ctx.fhs_set_dde(0, dd.kern, dd.kidx)
    out = {"workload": spec.name, "kernel": f"{S_d}x{S_d} DDE kernels, {7 + S_d - 1}x{7 + S_d - 1} footprints",
           "baselines": DDE_N_ANT * (DDE_N_ANT - 1) // 2, "visibilities_per_launch": int(spec.M * spec.Lc)}
    for name in ("degrid", "grid"):
        ctx.fhs_set_kernel_timer(name)
        ms = timed_iters(3)
        t, n = ctx.fhs_kernel_timer_read()
        ctx.fhs_set_kernel_timer(None)
        sec = t / n / 1000.0
        flops = dde_flops_per_vis(S_d) * spec.M * spec.Lc
        peak = 152 * 128 * 2 * (sm_mhz or 2070.0) * 1e6 / 1e12
        ach = flops / sec / 1e12
        out[name] = {"ms_per_launch": round(sec * 1e3, 3), "vis_per_s": round(spec.M * spec.Lc / sec, 1),
                     "roofline": {"bound": "alu", "achieved": round(ach, 2), "peak": round(peak, 1),
                                  "unit": "TFLOP/s", "frac": round(ach / peak, 4),
                                  "peak_kind": "derived: FP32 FMA lanes x 2 x sampled SM clock"}}
    out["iteration_ms"] = {"plain_rows": round(plain_ms, 3), "dde_rows": round(ms, 3)}
    ctx.close()
    # the oracle on a sample of the same rows (one channel, 4000 visibilities)
    K = 2 * spec.n
    g = np.random.default_rng(1).standard_normal((K, K)) + 0j
    uvs = (base[perm[:4000]]).astype(np.float32).astype(np.float64)
    kidx = dd.kidx[:4000]
    t0 = time.perf_counter()
    u = odde.degrid(g, uvs, dd.kern, kidx)
    odde.grid_adjoint(u, uvs, dd.kern, kidx, K, K)
    dt = time.perf_counter() - t0
    out["oracle"] = {"vis_per_s_degrid_plus_grid": round(4000 / dt, 1), "cores": 1,
                     "sample": "4000 visibilities of channel 0 on a 2048^2 grid, de-gridding then gridding"}
    return out


# ------------------------------------------------ mixed-size batch (Section 2.4.1)
def batch_measurement(args, torch, log) -> dict:
    """The mixed-size batch: 16 independent cubes of uneven shapes (sides 128..768, 3 * 2^m
    sides included; 8..48 channels; 1..6 facets a side; 0.3..2 visibilities per pixel) in
    one context, one CUDA graph per iteration over all of them.  Data y = Phi x + noise
    formed with the library; parameters from the noise levels on the device
    (fhs_heuristic_params); the launch choices of every shape measured by the autotuner
    when the context is created.  Times 1, 2 and 4 lanes (fhs_set_lanes) and reports the
    iterations per second of the whole batch with the fastest, and the choices per
    cube."""
    from paper_2003_07358_gb300.fhs import Context, CubeParams
    specs = fs.batch_specs()
    cps, skies = [], []
    for spec in specs:
        rng = np.random.default_rng(spec.seed)
        sources = fs.sky_sources(spec, rng)
        base = fs.base_uv(spec, rng)
        blocks = fs.radial_blocks(base, spec.B)
        perm = np.concatenate(blocks)
        chans = fs.subcube_channels(spec, 0)
        uv = np.concatenate([fs.channel_uv(base, spec, l)[perm] for l in chans])
        M_lb = np.array([[b.size for b in blocks]] * spec.L, dtype=np.int64)
        cps.append(CubeParams(n1=spec.n, n2=spec.n, L=spec.L, Qy=spec.Q, Qx=spec.Q, overlap=spec.overlap,
                              window=spec.window, M_lb=M_lb, uv=uv, eta=np.ones(spec.L), mu=0.0,
                              mu_bar=np.zeros(spec.Q * spec.Q), eps=np.zeros((spec.L, spec.B))))
        skies.append((sources, chans, M_lb))
    # the launch choices of every shape measured in fhs_create (autotuner, mode 2), then
    # the bench's own setting again
    from paper_2003_07358_gb300.fhs import fhs_set_autotune
    fhs_set_autotune(2, os.path.join(tempfile.gettempdir(), "fhs_autotune_batch.json"))
    t0 = time.time()
    try:
        ctx = Context(cps)
    finally:
        fhs_set_autotune(args.autotune, os.path.join(tempfile.gettempdir(), "fhs_autotune_rank0.json")
                         if args.autotune else None)
    ctx_s = time.time() - t0
    log(f"batch context ({len(specs)} cubes, autotuned) created in {ctx_s:.1f} s")
    dev = ctx.device
    gen = torch.Generator(device=dev)
    its = []
    for c, spec in enumerate(specs):
        sources, chans, M_lb = skies[c]
        x = torch.empty((spec.L, spec.n, spec.n), device=dev)
        for i, l in enumerate(chans):
            x[i].copy_(torch.from_numpy(fs.render_channel(spec, sources, int(l)).astype(np.float32)))
        sz = ctx.sizes(c)
        y = torch.empty(sz["n_vis"], dtype=torch.complex64, device=dev)
        ctx.fhs_measure(c, x, y)
        zero = torch.zeros_like(y)
        tmp = torch.empty_like(y)
        dn = ctx.fhs_proj_l2ball_blocks(c, y, zero, tmp).reshape(spec.L, spec.B)
        Ml = M_lb.sum(axis=1)
        sigma = np.sqrt((dn ** 2).sum(axis=1)) / np.sqrt(Ml) * 10 ** (-spec.isnr_db / 20)
        gen.manual_seed(spec.seed)
        off = 0
        for i in range(spec.L):
            m = int(Ml[i])
            y[off:off + m] += float(sigma[i]) * torch.randn(m, dtype=torch.complex64, device=dev, generator=gen)
            off += m
        ctx.fhs_heuristic_params(c, sigma, power_iters=10)
        X = torch.zeros_like(x)
        its.append({"X": X, "Xcheck": torch.zeros_like(X), "y": y, "state": ctx.new_state(c)})
        del x, zero, tmp
    stream = ctx.stream
    k = 5

    def timed(lanes):
        ctx.fhs_set_lanes(lanes)
        for _ in range(3):
            ctx.fhs_pdfb_iter(its, 1, want_stats=False)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            ctx.fhs_pdfb_iter(its, 1, want_stats=False)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    lane_ms = {n: round(timed(n), 3) for n in (1, 2, 4)}
    best = min(lane_ms, key=lane_ms.get)
    ms = timed(best)
    st = ctx.fhs_pdfb_iter(its, 1, want_stats=True)
    tuning = {}
    for c, spec in enumerate(specs):
        t = ctx.fhs_get_tuning(c)
        tuning[spec.name] = {kk: t[kk] for kk in ("grid_tile", "degrid_tiled", "gram_tc", "sara_fast",
                                                  "prox_ctas_per_sm", "source")}
    out = {"workload": "mixed-size batch: 16 cubes, sides 128..768 (3 * 2^m included), L 8..48, 1..6 facets a side, "
                       "M/N 0.3..2, B 1..4",
           "cubes": len(specs), "pixel_channels": int(sum(sp.n * sp.n * sp.L for sp in specs)),
           "visibilities": int(sum(sp.M * sp.L for sp in specs)), "ms_per_iteration": round(ms, 3),
           "iter_per_s": round(1000.0 / ms, 3), "lanes": ctx.fhs_get_lanes(), "timed_iterations": k,
           "ms_per_iteration_by_lanes": lane_ms, "context_and_autotune_s": round(ctx_s, 1),
           "xi_last": [round(s_["xi"], 6) for s_ in st], "choices_by_cube": tuning}
    ctx.close()
    log(f"batch: {ms:.2f} ms per iteration")
    return out


# ------------------------------------------------------- algorithmic bytes
def op_bytes(spec: fs.CubeSpec, n_coef: int, n_facet_pix: int) -> dict:
    """Algorithmic HBM bytes per sub-cube of each operator (each array read or
    written once, pruned FFT passes, FP32 / complex64)."""
    N = spec.n * spec.n
    L = spec.Lc
    M = spec.M
    return {
        "sara": 4 * N * L + 8 * n_coef * L + 4 * n_coef + 4 * N * L,
        "nuclear": 12 * n_facet_pix * L + 8 * N * L + 4 * N * L,
        "data": L * (200 * N + 32 * M),          # measure + adjoint
        "primal": 24 * N * L,
    }


def grid_launch_bytes(spec: fs.CubeSpec) -> int:
    """Algorithmic bytes of one gridding launch (one sub-cube): the 2n x 2n complex64
    grid of each channel written once, and per visibility uv (8 B), value (8 B), block
    id (1 B) read and the scaled dual v (8 B) written."""
    K2 = (2 * spec.n) ** 2
    return spec.Lc * (8 * K2 + 25 * spec.M)


# DRAM bytes (read + write) per channel of one gridding launch (k_grid<0>), measured by
# ncu on the large_slice workload (4096^2 image, 8192^2 grid, 8,388,608 visibilities per
# channel): dram__bytes_read.sum + dram__bytes_write.sum = 291.7 MB + 1147.9 MB for its 2
# channels (profiles/k_grid_large_slice_ncu.md).  Traffic scales with the channels of a
# launch (each channel's grid and visibilities are separate).
K_GRID_DRAM_BYTES_PER_CHANNEL = 719_793_664


def grid_traffic(spec: fs.CubeSpec):
    """DRAM traffic of one gridding launch from the measured per-channel figure; None on
    other workload geometries."""
    if spec.n == 4096 and spec.M == fs.workload("large_slice").M:
        return int(K_GRID_DRAM_BYTES_PER_CHANNEL * spec.Lc)
    return None


# --------------------------------------------------------- SNR gap vs FP64
GOLDEN = os.path.join(ROOT, "tests", "golden")


def snr_gaps(torch, log) -> dict:
    """Reconstruction SNR (Section 4.2) of the GPU path against the stored FP64 oracle runs
    of the tiny, faceted and reduced precision-form workloads (same seeded inputs, same
    parameters, same schedule);
    the data are formed with the library's own measurement operator."""
    from paper_2003_07358_gb300.fhs import Context, CubeParams
    out = {}
    runs = {"tiny": "tiny_pdfb_schedule.json", "faceted": "faceted_pdfb200.json",
            "precision_small": "precision_small_pdfb100.json"}
    for key, fname in runs.items():
        with open(os.path.join(GOLDEN, fname)) as f:
            rec = json.load(f)
        spec = fs.workload(rec["workload"], **rec["over"])
        inp = fs.make_inputs(spec)
        L, n = inp.x_true.shape[0], spec.n
        ctx = Context([CubeParams(n1=n, n2=n, L=L, Qy=spec.Q, Qx=spec.Q, overlap=spec.overlap, window=spec.window,
                                  M_lb=inp.M_lb, uv=inp.uv, eta=np.array(rec["eta"]), mu=rec["mu"],
                                  mu_bar=np.array(rec["mu_bar"]), eps=np.array(rec["eps"]), tau=rec["tau"],
                                  zeta=rec["zeta"], kappa=rec["kappa"])])
        xt = torch.as_tensor(inp.x_true.astype(np.float32), device="cuda")
        y = torch.empty(inp.uv.shape[0], dtype=torch.complex64, device="cuda")
        ctx.fhs_measure(0, xt, y)
        noise = np.zeros(inp.uv.shape[0], dtype=np.complex64)
        off = 0
        for l in range(L):
            m = int(inp.M_lb[l].sum())
            noise[off:off + m] = rec["sigma"][l] * inp.noise[off:off + m]
            off += m
        nz = torch.empty_like(y)
        ctx.fhs_vis_to_internal(0, torch.as_tensor(noise, device="cuda"), nz)
        y += nz
        X = torch.zeros_like(xt)
        st = ctx.new_state(0)
        it = [{"X": X, "Xcheck": torch.zeros_like(X), "y": y, "state": st}]
        for step in rec["schedule"]:
            if step == "reweight":
                ctx.fhs_reweight(0, X, st["theta"], st["theta_bar"])
            else:
                ctx.fhs_pdfb_iter(it, step, want_stats=False)
        Xg = X.double().cpu().numpy()
        snr = [20.0 * math.log10(np.linalg.norm(inp.x_true[l]) / np.linalg.norm(inp.x_true[l] - Xg[l]))
               for l in range(L)]
        ref = rec["snr_db"]
        shape = f"{spec.n}x{spec.n}, L={spec.L}, {spec.Q}x{spec.Q} facets, B={spec.B} ({rec['workload']} form)"
        out[key] = {"workload": shape, "schedule": rec["schedule"], "gpu_snr_db": round(float(np.mean(snr)), 4),
                    "oracle_snr_db": round(float(np.mean(ref)), 4),
                    "gap_db": round(float(np.mean(snr) - np.mean(ref)), 5),
                    "max_channel_gap_db": round(float(np.max(np.abs(np.array(snr) - ref))), 5)}
        ctx.close()
        log(f"SNR gap {key}: {out[key]}")
    out["precision_full_size"] = ("not measured: the oracle is too slow for 1024^2 x 32; the precision form's "
                                  "sky and channels are measured on 256^2 (precision_small)")
    return out


# ------------------------------------------------------------- CPU oracle
def oracle_iteration_estimate(spec: fs.CubeSpec, budget_scale: float = 1.0) -> dict:
    """Seconds of one oracle iteration of the workload, from timed samples of
    each operator scaled by the number of units per iteration."""
    from oracle import nufft as nu
    from oracle import prox as px
    from oracle import wavelets as wv
    rng = np.random.default_rng(11)
    n, Lc, C, Q = spec.n, spec.Lc, spec.C, spec.Q
    L = spec.L
    out = {}
    # data term: forward FFT of one channel + degrid / grid of a visibility sample
    x = rng.random((n, n))
    t = time.perf_counter()
    g = nu.zpad_fft(x)
    t_fft = time.perf_counter() - t
    ms = max(2000, int(20000 * budget_scale))
    uv = rng.uniform(-math.pi / 2, math.pi / 2, (ms, 2))
    t = time.perf_counter()
    y = nu.degrid(g, uv)
    t_deg = time.perf_counter() - t
    t = time.perf_counter()
    nu.grid_adjoint(y, uv, 2 * n, 2 * n)
    t_grd = time.perf_counter() - t
    per_ch = 2 * t_fft + (t_deg + t_grd) * spec.M / ms
    out["data"] = per_ch * L
    # SARA: analysis + synthesis of a crop, scaled by area and channels
    s = min(n, 1024 if budget_scale >= 4 else (512 if budget_scale >= 1 else 256))
    xs = rng.random((1, s, s))
    t = time.perf_counter()
    cf = wv.sara_analysis(xs)
    wv.sara_synthesis(cf, s, s)
    out["sara"] = (time.perf_counter() - t) * (n * n) / (s * s) * L
    # nuclear: Jacobi SVD of one facet-sized matrix, scaled by facets and sub-cubes
    side = n // Q + int(math.floor(spec.overlap * n / Q))
    rows = min(side * side, 32768 if budget_scale >= 4 else (8192 if budget_scale >= 1 else 4096))
    Z = rng.standard_normal((rows, Lc))
    t = time.perf_counter()
    px.jacobi_svd(Z)
    out["nuclear"] = (time.perf_counter() - t) * (side * side / rows) * Q * Q * C
    # primal: elementwise update of one channel
    X = rng.random((n, n))
    A = rng.random((n, n))
    t = time.perf_counter()
    Xn = px.proj_nonneg_real(X - 0.33 * A)
    _ = 2 * Xn - X
    out["primal"] = (time.perf_counter() - t) * L
    out["total"] = sum(out.values())
    return out


def oracle_faceted_iteration_seconds() -> float:
    """Wall time of one whole FP64 oracle PDFB iteration of the faceted workload (256^2,
    L = 20, 4 x 4 facets, 2 blocks): a measured unit, not an extrapolation."""
    from oracle import pdfb as pd
    spec = fs.workload("faceted")
    inp = fs.make_inputs(spec)
    prob, _ = pd.build_problem(inp, power_iters=2)      # parameters do not change the cost
    st = pd.initial_state(prob)
    pd.pdfb_iteration(prob, st)
    t = time.perf_counter()
    pd.pdfb_iteration(prob, st)
    return time.perf_counter() - t


def _estimate_worker(args):
    spec_name, scale = args
    return oracle_iteration_estimate(fs.WORKLOADS[spec_name], scale)["total"]


def oracle_all_cores(spec_name: str, scale: float, cores: int) -> dict:
    """The sampled estimate run by `cores` processes at once (spawned): the oracle's
    iteration is independent per channel, so all-core throughput = cores x the
    per-process rate measured under that load."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(cores) as pool:
        totals = pool.map(_estimate_worker, [(spec_name, scale)] * cores)
    per_iter = statistics.median(totals)               # seconds per iteration of one process
    return {"value": cores / per_iter, "unit": "iter/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} concurrent processes, each timing the sampled estimate; throughput = "
                      "processes / median seconds per iteration"}


def run_reference(args, spec):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    for _ in range(args.warmup):
        oracle_iteration_estimate(spec, 0.25)
    vals = []
    t0 = time.time()
    for _ in range(args.steps):
        est = oracle_iteration_estimate(spec, 0.25)
        vals.append(1.0 / est["total"])
    wall = time.time() - t0
    v = statistics.median(vals)
    anchor = oracle_faceted_iteration_seconds()
    sample = ("per step: one channel's 2n x 2n FFT, 5000 degrid + grid visibilities, SARA on a 256^2 crop, "
              "Jacobi SVD of a 4096 x 16 facet slice, one channel's primal update; each scaled to the "
              "units of one full iteration (an estimate: one iteration of this workload takes hours)")
    # a step is one bounded sample (its wall time is ms_per_step); value scales each
    # sample's operator times to one whole iteration of the workload (an estimate, with its
    # time per iteration stated separately)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "iter/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / max(args.steps, 1),
            "ms_per_iteration_estimate": 1000.0 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": spec.name, "oracle": "numpy float64"},
            "estimate": True,
            "measured_anchor": {"workload": fs.workload("faceted").name, "oracle_s_per_iteration": round(anchor, 3),
                                "what": "one whole FP64 oracle PDFB iteration, timed"},
            "cpu_baseline": {"value": v, "unit": "iter/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- main
def main():
    args = parse()
    spec = fs.WORKLOADS[args.workload]
    env_world = os.environ.get("WORLD_SIZE")
    if args.gpus > 1 and env_world is None:
        sys.exit(relaunch_under_torchrun(args))
    if env_world is not None and int(env_world) != args.gpus:
        sys.exit(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={env_world}")
    if args.dry_run:
        dry_run(args)
        return
    if args.impl == "reference":
        run_reference(args, spec)
        return
    import torch
    from paper_2003_07358_gb300 import sharding as sh
    info = sh.rank_info()
    rank, world, local = info.rank, info.world, info.local
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)

    def log(msg):
        if rank == 0:
            print(f"[bench] {msg}", file=sys.stderr, flush=True)

    import __graft_entry__
    __graft_entry__.build()
    if args.autotune:
        from paper_2003_07358_gb300.fhs import fhs_set_autotune
        fhs_set_autotune(args.autotune, os.path.join(tempfile.gettempdir(), f"fhs_autotune_rank{rank}.json"))
    ctx, its = setup(spec, torch, rank, args.opnorm_iters, log)
    ctx.fhs_set_lanes(args.lanes)
    tuning = {}
    for c in range(spec.C):
        t = ctx.fhs_get_tuning(c)
        key = f"{spec.n}x{spec.n} L={spec.Lc} Q={spec.Q}x{spec.Q} B={spec.B} M={spec.M}"
        tuning.setdefault(key, {k: t[k] for k in ("grid_tile", "degrid_tiled", "gram_tc", "sara_fast",
                                                  "prox_ctas_per_sm", "source")})
    stream = ctx.stream

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    # CUDA events around the gridding kernel inside the captured iteration (the
    # dominant kernel of the iteration), read after the timed region
    ctx.fhs_set_kernel_timer("grid")
    for _ in range(args.warmup):
        ctx.fhs_pdfb_iter(its, 1, want_stats=False)
    st = ctx.fhs_pdfb_iter(its, 1, want_stats=True)
    log(f"warm-up done, stats {st}")
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = ctx.fhs_kernel_launches()
    log(f"timed region starts after {l0} library kernel launches")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.fhs_pdfb_iter(its, 1, want_stats=False)
    e1.record(stream)
    barrier()
    launches = ctx.fhs_kernel_launches() - l0
    lanes = ctx.fhs_get_lanes()
    clocks = sampler.stop()
    grid_ms, grid_n = ctx.fhs_kernel_timer_read()
    ctx.fhs_set_kernel_timer(None)
    ms = sh.max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, device="cuda")
    value = sh.weak_scaling_value(1, world, ms / 1000.0)
    log(f"{ms:.1f} ms per iteration")

    # the plain FP32 path (one launch per pass, unfused) on the same state, for the speed-up
    plain = None
    if args.plain_steps > 0:
        ctx.fhs_set_path("plain")
        ctx.fhs_pdfb_iter(its, 1, want_stats=False)
        barrier()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(args.plain_steps):
            ctx.fhs_pdfb_iter(its, 1, want_stats=False)
        p1.record(stream)
        barrier()
        ctx.fhs_set_path("fast")
        pms = p0.elapsed_time(p1) / args.plain_steps
        plain = {"ms_per_step": pms, "value": world * 1000.0 / pms, "speedup_fast_over_unfused": pms / ms,
                 "what": ("FHS_PATH_PLAIN: the first, unfused FP32 kernels (SARA analysis, l2,1 dual and synthesis "
                          "as separate passes through a materialised coefficient array, untiled degridder, "
                          "CUDA-core float-float Grams), direct launches without a graph; the gridder, FFTs, "
                          "eigen-solve, nuclear update and primal kernels are shared with the fast path, so this "
                          "is not a fully independent plain implementation")}
        log(f"plain path {pms:.1f} ms per iteration")

    # per-operator times through their own C-ABI calls (same stream, CUDA events)
    hbm, peak_kind = peaks()
    ops = {}
    sz = ctx.sizes(0)
    if not args.no_ops:
        A = torch.zeros_like(its[0]["X"])
        ybuf = torch.empty_like(its[0]["y"])

        def time_op(fn, reps=3):
            fn()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps / 1000.0

        it0 = its[0]
        s0 = it0["state"]
        times = {
            "sara": time_op(lambda: ctx.fhs_prox_l21_sara_facets(0, it0["Xcheck"], s0["W"], s0["theta"], A)),
            "nuclear": time_op(lambda: ctx.fhs_prox_nuclear_facets(0, it0["Xcheck"], s0["P"], s0["theta_bar"], A)),
            "data": time_op(lambda: (ctx.fhs_measure(0, it0["X"], ybuf), ctx.fhs_adjoint(0, ybuf, A))),
        }
        byts = op_bytes(spec, sz["n_coef"], sz["n_facet_pix"])
        for k, t in times.items():
            gbs = byts[k] / t / 1e9
            ops[k] = {"ms_per_subcube": round(t * 1e3, 3), "algorithmic_GB": round(byts[k] / 1e9, 3),
                      "GB_s": round(gbs, 1), "frac_of_hbm": round(gbs / hbm, 4)}
        ops["primal"] = {"algorithmic_GB": round(byts["primal"] / 1e9, 3)}
        del A, ybuf
    # roofline of the dominant kernel, the gridder G^T: one launch grids one sub-cube,
    # algorithmic bytes = grid written once (L K1 K2 8 B) + per visibility uv, value,
    # block id read and v written (25 B); time = its CUDA events in the last timed iteration
    g_bytes = grid_launch_bytes(spec)
    g_s = grid_ms / grid_n / 1000.0
    g_ach = g_bytes / g_s / 1e9
    roofline = {"bound": "hbm", "kernel": "k_grid (gridding G^T, one sub-cube per launch)",
                "achieved": round(g_ach, 1), "peak": hbm, "unit": "GB/s", "frac": round(g_ach / hbm, 4),
                "traffic": grid_traffic(spec), "peak_kind": peak_kind,
                "ms_per_launch": round(g_s * 1e3, 3), "algorithmic_GB_per_launch": round(g_bytes / 1e9, 3)}

    # end to end through the C ABI with host buffers (fhs_pdfb_iter_host): every step copies
    # each sub-cube's data y from pinned host memory (caller's order) and the iterate X
    # back to pinned host memory, inside the timed region
    e2e = None
    if not args.no_e2e:
        y_hosts, x_hosts = [], []
        for c, it in enumerate(its):
            yu = torch.empty_like(it["y"])
            ctx.fhs_vis_to_user(c, it["y"], yu)
            y_hosts.append(yu.cpu().pin_memory())
            x_hosts.append(torch.empty(it["X"].shape, dtype=torch.float32).pin_memory())
            del yu
        h2d = sum(h.numel() * 8 for h in y_hosts)
        d2h = sum(h.numel() * 4 for h in x_hosts)
        k = max(2, args.steps // 2)
        ctx.fhs_pdfb_iter_host(its, y_hosts, x_hosts, 1, want_stats=False)
        barrier()
        t0 = time.perf_counter()
        for _ in range(k):
            ctx.fhs_pdfb_iter_host(its, y_hosts, x_hosts, 1, want_stats=False)
        barrier()
        ems = (time.perf_counter() - t0) * 1000.0 / k
        e2e = {"value": world * 1000.0 / ems, "unit": "iter/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "call": "fhs_pdfb_iter_host (y from pinned host memory, X back to pinned host memory, synchronising)"}
        del y_hosts, x_hosts

    gaps = None
    if rank == 0 and world == 1 and not args.no_snr_gap:
        gaps = snr_gaps(torch, log)

    dde_line = None
    if rank == 0 and world == 1 and not args.no_dde:
        dde_line = dde_measurement(args, torch, log, clocks.get("sm_mhz"))

    batch_line = None
    if rank == 0 and world == 1 and not args.no_batch:
        batch_line = batch_measurement(args, torch, log)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t = time.time()
        est = oracle_iteration_estimate(spec, 4.0)
        cpu = {"value": 1.0 / est["total"], "unit": "iter/s", "cores": 1, "kind": "oracle",
               "sample": ("one channel's 2n x 2n FFT, 80000 degrid + grid visibilities, SARA on a 1024^2 crop, "
                          "Jacobi SVD of a 32768 x 16 facet slice, one channel's primal update, each scaled "
                          "to the units of one full iteration; seconds per iteration by operator: "
                          + ", ".join(f"{k} {v:.0f}" for k, v in est.items())),
               "wall_s": round(time.time() - t, 1)}
        cores = os.cpu_count() or 1
        if cores > 1:
            cpu["all_cores"] = oracle_all_cores(args.workload, 1.0, cores)
        cpu["measured_anchor"] = {"workload": fs.workload("faceted").name,
                                  "oracle_s_per_iteration": round(oracle_faceted_iteration_seconds(), 3)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": spec.name, "n": spec.n, "L": spec.L, "subcubes": spec.C,
                           "facets": f"{spec.Q}x{spec.Q}", "vis_per_channel": spec.M, "blocks": spec.B,
                           "path": "FP32 fused kernels (FP64 reductions)", "lanes": lanes,
                           "l2": "working set ~100 GB >> 129 MB L2; no flush"},
                "roofline": roofline, "operators": ops, "cpu_baseline": cpu, "e2e": e2e,
                "plain_fp32_path": plain, "snr_gap_vs_fp64": gaps, "dde_degridding": dde_line, "mixed_size_batch": batch_line,
                "clocks": clocks,
                "autotune_by_shape": tuning, "gpu_launches": launches}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
