"""Continuous-batching server: a job's result is the same alone and in a
mix of concurrent jobs (bitwise), admission respects the HBM budget, and
the plain per-step-launch server agrees."""
import numpy as np
import pytest

from gpu_helpers import I, torch  # noqa: F401

import paper_2412_16490_gb300 as bx
from paper_2412_16490_gb300.serving import JobSpec, PlainServer, Server, job_bytes, object_bytes

pytestmark = pytest.mark.gpu


def _specs():
    T = I.wrench_set(12)
    objs = [I.grid_object(41, n=32, h=0.128 / 31), I.sphere_object(), I.grid_object(42, n=48, h=0.128 / 47)]
    out = []
    for k, (name, oi, B, n) in enumerate((("hand5", 0, 40, 20), ("hand3", 1, 17, 15), ("hand4x4", 2, 64, 25),
                                           ("hand5", 2, 9, 10), ("hand3", 0, 33, 20))):
        hand = I.hand_template(name)
        x0 = I.initial_poses(hand, objs[oi], B, seed=60 + k)
        out.append(JobSpec(hand, objs[oi], x0, T, n, arrival=0.002 * k, tag=k))
    return out


P = I.default_params()
QP = bx.qp_params(max_iter=20)


def test_job_result_is_the_same_alone_and_in_the_mix():
    specs = _specs()
    mix = Server(P, qp=QP, steps_per_tick=4).replay(specs, realtime=False)
    for k, sp in enumerate(specs):
        alone = Server(P, qp=QP, steps_per_tick=4).replay([sp], realtime=False)[0]
        assert np.array_equal(mix[k].x, alone.x), k
        assert np.array_equal(mix[k].E, alone.E), k


def test_admission_respects_the_hbm_budget():
    specs = _specs()
    need = [job_bytes(s) for s in specs]
    grids = sum(object_bytes(o) for o in {id(s.obj): s.obj for s in specs}.values())
    budget = max(job_bytes(s) + object_bytes(s.obj) for s in specs) + 1  # the largest job fits alone
    srv = Server(P, qp=QP, steps_per_tick=5, hbm_budget=budget)
    res = srv.replay(specs, realtime=False)
    assert len(res) == len(specs) and srv.used == 0
    assert srv.peak_used <= budget and srv.peak_active < len(specs)
    free = Server(P, qp=QP, steps_per_tick=5, hbm_budget=sum(need) + grids).replay(specs, realtime=False)
    for k in res:
        assert np.array_equal(res[k].x, free[k].x)
    with pytest.raises(MemoryError):
        Server(P, qp=QP, hbm_budget=16).replay(specs[:1], realtime=False)


def test_plain_server_agrees_and_latencies_are_recorded():
    specs = _specs()
    cont = Server(P, qp=QP, steps_per_tick=5).replay(specs, realtime=True)
    plain = PlainServer(P, qp=QP).replay(specs, realtime=True)
    for k in cont:
        np.testing.assert_allclose(cont[k].x, plain[k].x, atol=1e-6)
        assert cont[k].latency > 0 and plain[k].latency > 0
        assert cont[k].finish >= cont[k].arrival
