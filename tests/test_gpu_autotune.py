"""The autotuner (fhs_set_autotune / fhs_get_tuning): choices measured per shape in
fhs_create, written to the JSON cache and read back for the same shape; defaults when
it is off; and every alternative it can choose (32-cell gridder tiles with the
tile-staged or the direct de-gridder, the CUDA-core Gram, the separate SARA passes, a
different CTA count of the l2,1 pass) giving the oracle's PDFB iterates."""
from __future__ import annotations

import json

import numpy as np
import pytest

from oracle import pdfb as pd

from _fixtures import make_context, make_problem, rel_err, vis_to_internal

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = [("tiny", {}), ("faceted", dict(n=128, L=6, Q=2, m_ratio=0.5, B=2))]


@pytest.fixture(autouse=True)
def _gpu_and_reset():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2003_07358_gb300.fhs import fhs_set_autotune
    yield
    fhs_set_autotune(0)


def test_measures_then_reads_the_cache(tmp_path):
    from paper_2003_07358_gb300.fhs import fhs_set_autotune
    path = str(tmp_path / "tune.json")
    fhs_set_autotune(1, path)
    for name, over in SHAPES:
        spec, inp, prob = make_problem(name, **over)
        ctx = make_context(prob, torch)
        t = ctx.fhs_get_tuning(0)
        ctx.close()
        assert t["source"] == "measured"
        assert t["grid_tile"] in (32, 64) and t["prox_ctas_per_sm"] in (4, 8, 16)
        assert all(v > 0 for v in t["ms"][:10]), t["ms"]
        # the measured times decide
        assert t["grid_tile"] == (32 if t["ms"][0] < t["ms"][1] else 64)
        assert t["degrid_tiled"] == int(t["ms"][2] <= t["ms"][3])
        assert t["gram_tc"] == int(t["ms"][4] <= t["ms"][5])
        ctx = make_context(prob, torch)
        t2 = ctx.fhs_get_tuning(0)
        ctx.close()
        assert t2["source"] == "cache"
        for k in ("grid_tile", "degrid_tiled", "gram_tc", "sara_fast", "prox_ctas_per_sm"):
            assert t2[k] == t[k]
    with open(path) as f:
        data = json.load(f)
    assert len(data) == 2
    # mode 2 measures again although the cache has the shape
    fhs_set_autotune(2, path)
    spec, inp, prob = make_problem(*SHAPES[0][:1], **SHAPES[0][1])
    ctx = make_context(prob, torch)
    assert ctx.fhs_get_tuning(0)["source"] == "measured"
    ctx.close()


def test_defaults_when_off():
    spec, inp, prob = make_problem("tiny")
    ctx = make_context(prob, torch)
    t = ctx.fhs_get_tuning(0)
    ctx.close()
    assert t["source"] == "defaults"
    assert (t["grid_tile"], t["degrid_tiled"], t["gram_tc"], t["sara_fast"], t["prox_ctas_per_sm"]) == (64, 1, 1, 1, 16)


FORCED = [
    dict(grid_tile=32, degrid_tiled=1, gram_tc=0, sara_fast=1, prox_ctas_per_sm=4),
    dict(grid_tile=32, degrid_tiled=0, gram_tc=1, sara_fast=0, prox_ctas_per_sm=16),
    dict(grid_tile=64, degrid_tiled=0, gram_tc=0, sara_fast=0, prox_ctas_per_sm=8),
]


@pytest.mark.parametrize("forced", FORCED, ids=["t32-tiled-ccgram", "t32-direct-plainsara", "t64-direct-ccgram"])
def test_every_choice_matches_the_oracle(tmp_path, forced):
    from paper_2003_07358_gb300.fhs import fhs_set_autotune
    path = str(tmp_path / "tune.json")
    name, over = SHAPES[1]
    spec, inp, prob = make_problem(name, **over)
    fhs_set_autotune(1, path)
    make_context(prob, torch).close()               # writes the measured entry
    with open(path) as f:
        data = json.load(f)
    (key,) = data
    data[key].update(forced)
    with open(path, "w") as f:
        json.dump(data, f)
    ctx = make_context(prob, torch)
    t = ctx.fhs_get_tuning(0)
    assert t["source"] == "cache"
    for k, v in forced.items():
        assert t[k] == v
    X = torch.zeros((prob.L, prob.n1, prob.n2), device="cuda")
    it = [{"X": X, "Xcheck": torch.zeros_like(X), "y": vis_to_internal(ctx, torch, prob.y), "state": ctx.new_state(0)}]
    n_iter = 6
    stats = ctx.fhs_pdfb_iter(it, n_iter)
    ctx.fhs_reweight(0, it[0]["X"], it[0]["state"]["theta"], it[0]["state"]["theta_bar"])
    stats = ctx.fhs_pdfb_iter(it, 2)
    st = pd.initial_state(prob)
    for _ in range(n_iter):
        pd.pdfb_iteration(prob, st)
    st.theta, st.theta_bar = pd.reweight(prob, st.X)
    for _ in range(2):
        out = pd.pdfb_iteration(prob, st)
    assert rel_err(it[0]["X"].double().cpu().numpy(), st.X) < 1e-4
    assert stats[0]["xi"] == pytest.approx(out["xi"], rel=2e-3)
    ctx.close()


def test_corrupt_cache_entry_is_refused(tmp_path):
    from paper_2003_07358_gb300.fhs import FhsError, fhs_set_autotune
    path = str(tmp_path / "tune.json")
    spec, inp, prob = make_problem("tiny")
    fhs_set_autotune(1, path)
    make_context(prob, torch).close()
    with open(path) as f:
        data = json.load(f)
    (key,) = data
    data[key]["grid_tile"] = 48
    with open(path, "w") as f:
        json.dump(data, f)
    with pytest.raises(FhsError, match="INVALID_ARG"):
        make_context(prob, torch)
    # an unreadable file reads as empty: measured again and rewritten
    with open(path, "w") as f:
        f.write("{not json")
    ctx = make_context(prob, torch)
    assert ctx.fhs_get_tuning(0)["source"] == "measured"
    ctx.close()
    assert np.isfinite(json.load(open(path))[key]["ms_0"])
