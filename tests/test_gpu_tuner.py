"""The slab-inverse autotuner of the interface solve: a handle measures every
admissible variant on its first solve, writes its choice to the cache named by
MRCM_TUNE_CACHE, and a second handle of the same shape class takes the choice
from the cache and reproduces the first handle's solution bit for bit."""
import json

import numpy as np
import pytest

from paper_2404_13811_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _run(case):
    from paper_2404_13811_gb300 import _lib as L
    from paper_2404_13811_gb300.solver import MRCM
    pm = case.params
    s = MRCM(case.problem, case.partition, space=pm.space, alpha_basis=pm.alpha_basis,
             alpha_smooth=pm.alpha_smooth, precision="mixed")
    s.run(1)
    st = L.mrcm_stats(s.h)
    p, u = s.fluxes()
    s.close()
    return st, p, u


def test_tuning_cache_round_trip(tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("MRCM_TUNE_CACHE", str(cache))
    case = I.config_channel2d(n=128, n_smooth=1)
    st1, p1, u1 = _run(case)
    assert st1["slab_inverse_source"] == "measured", st1
    assert min(st1["tune_ms"].values()) > 0, st1   # all three slab inverses admit 128 x 128
    entries = json.loads(cache.read_text())
    assert len(entries) == 1
    (key, entry), = entries.items()
    assert key.startswith("interface dim2 ") and entry["slab_inverse"] == st1["slab_inverse"], (key, entry)
    assert entry["gauss_jordan_steps"] > 0 and entry["lu_steps"] > 0 and entry["gauss_jordan_registers_steps"] > 0
    st2, p2, u2 = _run(case)
    assert st2["slab_inverse_source"] == "cache" and st2["slab_inverse"] == st1["slab_inverse"], st2
    assert np.array_equal(p1, p2) and np.array_equal(u1, u2)


def test_metrics_line_per_outermost_call(tmp_path, monkeypatch):
    """MRCM_METRICS: one JSON line per outermost solve-path call, with the
    refinement counters and the slab-inverse choice; mrcm_run's inner calls
    write none."""
    log = tmp_path / "metrics.jsonl"
    monkeypatch.setenv("MRCM_METRICS", str(log))
    monkeypatch.delenv("MRCM_TUNE_CACHE", raising=False)
    from paper_2404_13811_gb300.solver import MRCM
    case = I.config_channel2d(n=128, n_smooth=1)
    pm = case.params
    s = MRCM(case.problem, case.partition, space=pm.space, alpha_basis=pm.alpha_basis,
             alpha_smooth=pm.alpha_smooth, precision="mixed")
    s.run(1)
    s.build_basis()
    s.solve_interface()
    s.smooth(2)
    s.close()
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    assert [x["call"] for x in lines] == ["mrcm_run", "mrcm_build_basis", "mrcm_solve_interface", "mrcm_smooth"]
    assert all(x["rc"] == 0 and x["wall_ms"] > 0 for x in lines)
    si = lines[2]
    assert si["interface_ir_steps"] > 0 and 0 < si["interface_residual"] <= 1e-9, si
    assert si["slab_inverse"] in ("gauss-jordan", "lu", "gauss-jordan-registers") and si["subdomains"] == 64
    assert lines[3]["smooth_steps"] == 2
