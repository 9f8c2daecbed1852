"""Autotuner of the fused step (S-PK): it times every (tile, schedule)
candidate, returns the fastest one its rule accepts, caches the choice, and
the tuned parameters reproduce the run it measured."""
import numpy as np
import pytest

from gpu_helpers import I, cuda, torch

import paper_2412_16490_gb300 as bx
from paper_2412_16490_gb300 import autotune as AT

pytestmark = pytest.mark.gpu

SCHEDULES = (dict(mode="fixed", iters=10), dict(mode="fixed", iters=30),
             dict(mode="converge", eps=1e-5, check=25, cap=400), dict(mode="exact", cap=64))
TILES = (2, 8)


def _workload():
    hand, obj, x0, T, P, _, _ = I.workload("tiny", batch=64)
    return bx.Hand(hand), bx.Object(obj), cuda(x0), cuda(T), P


@pytest.mark.parametrize("residual", [None, 1e-5])
def test_autotune_picks_fastest_accepted_and_reproduces_it(residual):
    AT._cache.clear()
    H, Ob, x0, T, P = _workload()
    steps = 6
    out = AT.autotune(H, Ob, x0, T, P, steps=steps, reps=1, tiles=TILES, schedules=SCHEDULES,
                      reference=dict(mode="fixed", iters=30), residual=residual)
    table = out["table"]
    assert len(table) == len(TILES) * len(SCHEDULES)
    assert all(np.isfinite(t["ms"]) and t["ms"] > 0 and np.isfinite(t["median_E"]) for t in table)
    ok = [t for t in table if t["ok"]]
    pool = ok or table
    best = min(pool, key=lambda t: t["ms"])
    assert out["ms"] == best["ms"] and out["grasps_per_cta"] == best["tile"] and out["schedule"] == best["schedule"]
    if residual is None:
        # the reference schedule (30 iterations) meets its own energy rule
        assert any(t["ok"] and t["schedule"] == dict(mode="fixed", iters=30) for t in table)
    else:
        for t in table:
            assert t["ok"] == (t["frac_res_le_1e5"] >= 0.99)
    # the tuned parameters run the chosen candidate: same final energies as the tuner saw
    st = bx.State(H, x0.shape[0], T.shape[0])
    st.set_pose(x0)
    E = torch.empty(x0.shape[0], device="cuda")
    bx.bodex_step(H, Ob, st, T, steps, AT.tuned_params(out, P), E_last=E)
    torch.cuda.synchronize()
    assert float(E.median().item()) == out["median_E"]
    # a second call with the same key returns the cached choice without timing again
    assert AT.autotune(H, Ob, x0, T, P, steps=steps, reps=1, tiles=TILES, schedules=SCHEDULES,
                       residual=residual) is out
