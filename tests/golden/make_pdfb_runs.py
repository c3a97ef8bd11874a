"""Writes the stored oracle runs that the GPU end-to-end tests compare against.

Runs only the FP64 oracle (``oracle/``) on the seeded synthetic inputs of
``fhs_synth``: the oracle is too slow to run these schedules inside a GPU test.

* ``tiny_pdfb_schedule.json``: 64 x 64, L = 4, Q = 1, M = 2000, B = 1, iSNR 40 dB;
  200 PDFB iterations (Algorithm 2) with unit weights, one weight update
  (Algorithm 1, Eqs. 9-10), 200 more iterations.
* ``faceted_pdfb200.json``: 256 x 256, L = 20, 4 x 4 facets, 10 % sine overlap,
  M = 0.5 N in 2 blocks, iSNR 40 dB; 200 PDFB iterations with unit weights.
* ``precision_small_pdfb100.json``: the precision form's sky, channels and noise (L = 32,
  Gaussian and point sources with 1 % spectral curvature, M = N in 4 blocks, iSNR 30 dB)
  on 256 x 256 with 4 x 4 facets; 100 PDFB iterations with unit weights.

Each file holds the parameters the oracle computed (sigma, eps, eta, mu, mu_bar), so the
GPU side uses exactly the oracle's values, and the results: per-channel SNR
(Section 4.2), xi and ||r|| of the last iteration, and X at seeded sampled pixels.

Usage: python tests/golden/make_pdfb_runs.py [tiny|faceted|precision_small ...]
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import fhs_synth as fs  # noqa: E402
from oracle import pdfb as pd  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
RUNS = {
    "tiny": dict(workload="tiny", over={}, power_iters=100, schedule=[200, "reweight", 200],
                 file="tiny_pdfb_schedule.json"),
    "faceted": dict(workload="faceted", over={}, power_iters=60, schedule=[200],
                    file="faceted_pdfb200.json"),
    "precision_small": dict(workload="precision", over={"n": 256, "Q": 4, "n_blobs": 60, "n_points": 60},
                            power_iters=40, schedule=[100], file="precision_small_pdfb100.json"),
}
N_SAMPLES = 128          # sampled pixels per channel


def run(name: str) -> None:
    cfg = RUNS[name]
    t0 = time.time()
    spec = fs.workload(cfg["workload"], **cfg["over"])
    inp = fs.make_inputs(spec)
    prob, aux = pd.build_problem(inp, power_iters=cfg["power_iters"])
    # both sides iterate on the complex64 data the GPU holds
    prob.y = prob.y.astype(np.complex64).astype(np.complex128)
    st = pd.initial_state(prob)
    done = 0
    out = None
    for step in cfg["schedule"]:
        if step == "reweight":
            st.theta, st.theta_bar = pd.reweight(prob, st.X)
            continue
        for _ in range(step):
            out = pd.pdfb_iteration(prob, st)
            done += 1
        print(f"[{name}] {done} iterations, {time.time() - t0:.0f} s", flush=True)
    rng = np.random.default_rng(12345)
    L, n1, n2 = prob.L, prob.n1, prob.n2
    pix = rng.choice(n1 * n2, size=(L, N_SAMPLES), replace=False if n1 * n2 >= N_SAMPLES else True)
    # half of the samples on the brightest pixels of each channel, where X is non-zero
    for l in range(L):
        top = np.argsort(-st.X[l].ravel(), kind="stable")[: N_SAMPLES // 2]
        pix[l, : N_SAMPLES // 2] = top
    vals = np.stack([st.X[l].ravel()[pix[l]] for l in range(L)])
    rec = {
        "what": f"oracle run of workload '{cfg['workload']}' ({spec.name}), schedule {cfg['schedule']}",
        "written_by": "tests/golden/make_pdfb_runs.py (FP64 oracle only)",
        "workload": cfg["workload"], "over": cfg["over"], "schedule": cfg["schedule"],
        "power_iters": cfg["power_iters"],
        "sigma": aux["sigma"].tolist(), "opnorm_sq": aux["opnorm_sq"].tolist(),
        "eta": prob.eta.tolist(), "eps": prob.eps.tolist(), "mu": prob.mu, "mu_bar": prob.mu_bar.tolist(),
        "tau": prob.tau, "zeta": prob.zeta, "kappa": prob.kappa,
        "snr_db": pd.snr_db(inp.x_true, st.X).tolist(),
        "xi_last": out["xi"], "res_norm_last": float(np.linalg.norm(out["res"])),
        "x_norm": np.linalg.norm(st.X.reshape(L, -1), axis=1).tolist(),
        "sample_pixels": pix.tolist(), "sample_values": vals.tolist(),
        "oracle_seconds": round(time.time() - t0, 1),
    }
    with open(os.path.join(HERE, cfg["file"]), "w") as f:
        json.dump(rec, f, indent=0)
    print(f"[{name}] wrote {cfg['file']} in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    for name in (sys.argv[1:] or list(RUNS)):
        run(name)
