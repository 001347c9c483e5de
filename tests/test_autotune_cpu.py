"""Host logic of the launch-configuration tuner (no GPU): which configuration
it keeps for given timings.  The timed calls are replaced by a table of
times keyed on the option tried and on whether the whole batch or a probe
was timed, so the rules themselves are checked: the default survives
differences within the margin, the placement is re-timed on the whole batch
when that is cheap, and a cached choice is returned without timing."""
import types

import numpy as np
import pytest
import torch

from paper_1101_5803_gb300 import autotune

N_ALL = 1024


def _batch():
    geom = types.SimpleNamespace(nx=64, ny=64, sx=32, sy=32, kpsf=9, subpix=1, reg=2)
    probs = [types.SimpleNamespace(geom=geom), types.SimpleNamespace(geom=geom)]
    lens = torch.zeros((N_ALL, 7), dtype=torch.float64)
    lambdas = torch.ones((N_ALL, 16), dtype=torch.float64)
    return probs, lens, np.zeros(N_ALL, np.int32), lambdas, np.full(N_ALL, 16, np.int32)


def _fake_time(table, calls):
    def fake(ctx, probs, lens, prob_idx, lam, nl, reps, **kw):
        whole = int(lens.shape[0]) == N_ALL
        calls.append((whole, kw.get("variant"), kw.get("inner_eta"), kw.get("place")))
        if "place" in kw:
            return table[("full" if whole else "probe", kw["place"])]
        if "inner_eta" in kw:
            return table.get(("eta", kw["inner_eta"]), 100.0)
        return table.get(("variant", kw["variant"]), 100.0)
    return fake


@pytest.fixture
def tuner(tmp_path, monkeypatch):
    monkeypatch.setenv("MIRAGE_TUNE_CACHE", str(tmp_path / "tune.json"))
    ctx = types.SimpleNamespace(precision=autotune.MIRAGE_FP32)
    return ctx


def test_whole_batch_timing_decides_the_placement(tuner, monkeypatch):
    # on the probe the split placement (2) looks best; on the whole batch the
    # split placement with two CTAs per SM (5) is 6% faster than the default
    table = {("probe", p): t for p, t in {0: 100.0, 1: 101.0, 2: 90.0, 3: 120.0, 4: 110.0, 5: 99.0}.items()}
    table.update({("full", p): t for p, t in {0: 3558.0, 1: 3560.0, 2: 3620.0, 3: 4000.0, 4: 3900.0,
                                               5: 3353.0}.items()})
    calls = []
    monkeypatch.setattr(autotune, "_time", _fake_time(table, calls))
    cfg = autotune.tune_config(tuner, *_batch())
    assert cfg == {"variant": 0, "inner_eta": autotune.ETAS[0], "place": 5}
    # every placement was timed on the whole batch, the default first
    whole = [c[3] for c in calls if c[0]]
    assert whole == [0] + list(autotune.PLACES)
    # a second call reads the cache and times nothing
    calls.clear()
    assert autotune.tune_config(tuner, *_batch()) == cfg
    assert calls == []


def test_expensive_batches_keep_the_probe_choice(tuner, monkeypatch):
    table = {("probe", p): t for p, t in {0: 100.0, 1: 101.0, 2: 90.0, 3: 120.0, 4: 110.0, 5: 99.0}.items()}
    table[("full", 0)] = autotune.FULL_BATCH_MS * 2
    calls = []
    monkeypatch.setattr(autotune, "_time", _fake_time(table, calls))
    cfg = autotune.tune_config(tuner, *_batch())
    assert cfg["place"] == 2
    assert [c[3] for c in calls if c[0]] == [0]  # only the cost check ran on the whole batch


def test_differences_within_the_margin_keep_the_defaults(tuner, monkeypatch):
    # every alternative within 2% of the default (below MARGIN = 3%)
    table = {("variant", v): 100.0 - v * 0.4 for v in autotune.VARIANTS}
    table.update({("eta", e): 100.0 - 1.5 * i for i, e in enumerate(autotune.ETAS)})
    table.update({("probe", p): 100.0 - 0.3 * p for p in (0,) + autotune.PLACES})
    table.update({("full", p): 3000.0 - 10.0 * p for p in (0,) + autotune.PLACES})
    monkeypatch.setattr(autotune, "_time", _fake_time(table, []))
    assert autotune.tune_config(tuner, *_batch()) == {"variant": 0, "inner_eta": autotune.ETAS[0], "place": 0}


def test_pick_rule():
    assert autotune._pick({0: 100.0, 1: 96.0}, 0) == 1
    assert autotune._pick({0: 100.0, 1: 97.5}, 0) == 0
    assert autotune._pick({0: 100.0, 1: 96.0}, 0, margin=0.05) == 0
