"""Host-side logic of the serving loop (no GPU): byte accounting and the
seeded Poisson workload."""
import numpy as np

import bodex_inputs as I
from paper_2412_16490_gb300.serving import JobSpec, PoissonWorkload, job_bytes, object_bytes


def test_job_bytes_counts_the_resident_state():
    hand = I.hand_template("hand5")
    spec = JobSpec(hand, I.sphere_object(), np.zeros((100, hand.dof), np.float32), I.wrench_set(12))
    D, m, s = hand.dof, 5, 12
    assert job_bytes(spec) == 4 * (100 * (3 * D + s * 12 * m + s + 2) + s * 6)
    assert object_bytes(I.sphere_object()) == 0
    g = I.grid_object(1, n=16, h=0.008)
    assert object_bytes(g) == 4 * 16 ** 3


def test_poisson_workload_is_seeded_and_has_the_requested_rate():
    a = PoissonWorkload(n_jobs=40, rate=20.0, seed=5, grid_choices=(16, 24)).build()
    b = PoissonWorkload(n_jobs=40, rate=20.0, seed=5, grid_choices=(16, 24)).build()
    assert [s.arrival for s in a] == [s.arrival for s in b]
    assert all(np.array_equal(x.x0, y.x0) for x, y in zip(a, b))
    gaps = np.diff([0.0] + [s.arrival for s in a])
    assert 0.02 < gaps.mean() < 0.09  # mean 1/20 s
    assert {s.tag["template"] for s in a} <= {"hand3", "hand4x4", "hand5"}
    assert all(s.x0.shape[0] in (256, 512, 1024, 2048, 4096) for s in a)


# ---- admission (Server._admit) on the host: the device-facing parts are stubbed
import types  # noqa: E402

import pytest  # noqa: E402

import paper_2412_16490_gb300 as bx  # noqa: E402
from paper_2412_16490_gb300.serving import Server, _Active, _Base, state_bytes  # noqa: E402

WAVE = 152 * 4  # thread blocks resident at once on a 152-SM GB300 (4 per SM)


def _host_server(hbm_budget=1 << 40, cta_budget=WAVE, max_jobs=64):
    """A Server without a device: what _admit reads and writes, with _open
    replaced by a stub that only registers the job's object."""
    srv = Server.__new__(Server)
    _Base.__init__(srv, I.default_params())
    srv.hbm_budget, srv.cta_budget, srv.ctas, srv.max_jobs = hbm_budget, cta_budget, 0, max_jobs
    srv.active, srv.finishing, srv.used, srv.pool, srv.pooled = [], [], 0, {}, 0
    srv.peak_active = srv.peak_used = 0

    def fake_open(jid, spec):
        srv._objects.setdefault(id(spec.obj), [None, 0])[1] += 1
        return _Active(jid, spec, None, None, None, None, None, spec.n_steps, 0.0, 0)

    srv._open = fake_open
    return srv


def _spec(B, tpl="hand5", obj=None, s=12):
    hand = I.hand_template(tpl)
    T = I.wrench_set(12)[:s].copy()
    return JobSpec(hand, obj if obj is not None else I.sphere_object(), np.zeros((B, hand.dof), np.float32), T)


def _finish(srv, a):
    """What tick/_reap do for a finished job, minus the device."""
    srv.active.remove(a)
    srv.ctas -= srv._job_ctas(a.spec)
    srv.used -= a.nbytes + srv._release_object(a.spec.obj)


def test_step_tile_is_the_kernel_tile():
    # 96 lanes / s, capped by the shared memory of one block for small s
    assert [bx.bodex_step_tile(5, s) for s in (6, 7, 12, 16)] == [16, 13, 8, 6]
    assert bx.bodex_step_tile(5, 12, 4) == 4 and bx.bodex_step_tile(5, 12, 100) == 8
    assert bx.bodex_step_tile(5, 1) < 96  # shared memory, not lanes, bounds it
    with pytest.raises(bx.BodexError):
        bx.bodex_step_tile(6, 12)
    with pytest.raises(bx.BodexError):
        bx.bodex_step_tile(5, 0)


def test_admission_is_fifo_within_one_wave_of_thread_blocks():
    srv = _host_server()
    big, mid, small = _spec(4096), _spec(1024), _spec(256)  # 512, 128, 32 blocks
    ids = [srv.submit(x) for x in (big, mid, small)]
    srv._admit()
    # 512 + 128 > 608: the second job waits, and the third behind it (FIFO)
    assert [a.jid for a in srv.active] == ids[:1] and srv.ctas == 512
    _finish(srv, srv.active[0])
    srv._admit()
    assert [a.jid for a in srv.active] == ids[1:] and srv.ctas == 160


def test_a_job_larger_than_a_wave_runs_alone():
    srv = _host_server()
    huge, small = _spec(8192), _spec(256)  # 1024 blocks, more than one wave
    ids = [srv.submit(huge), srv.submit(small)]
    srv._admit()
    assert [a.jid for a in srv.active] == ids[:1]
    _finish(srv, srv.active[0])
    srv._admit()
    assert [a.jid for a in srv.active] == ids[1:]


def test_admission_counts_bytes_and_shares_objects():
    grid = I.grid_object(3, n=16, h=0.008)
    a, b = _spec(256, obj=grid), _spec(256, obj=grid)
    obj_b = 4 * 16 ** 3
    srv = _host_server(hbm_budget=2 * job_bytes(a) + obj_b)  # the grid is counted once
    srv.submit(a), srv.submit(b)
    srv._admit()
    assert len(srv.active) == 2 and srv.used == 2 * job_bytes(a) + obj_b
    srv2 = _host_server(hbm_budget=2 * job_bytes(a) + obj_b - 1)
    srv2.submit(_spec(256, obj=grid)), srv2.submit(_spec(256, obj=grid))
    srv2._admit()
    assert len(srv2.active) == 1  # the second waits for memory
    with pytest.raises(MemoryError):
        srv3 = _host_server(hbm_budget=job_bytes(a) - 1)
        srv3.submit(_spec(256))
        srv3._admit()


def test_max_jobs_per_launch():
    srv = _host_server(max_jobs=2)
    for _ in range(3):
        srv.submit(_spec(64))
    srv._admit()
    assert len(srv.active) == 2 and len(srv._waiting) == 1


def test_pooled_states_are_reused_or_evicted():
    a = _spec(512)
    sb = state_bytes(a)
    fake_state = types.SimpleNamespace(B=512, D=a.hand.dof, s=12, m=5)
    # a pooled state of the job's shape: its bytes are already held, so the job fits
    srv = _host_server(hbm_budget=job_bytes(a))
    srv.pool = {(id(a.hand), 512, 12): [fake_state]}
    srv.pooled = sb
    srv.submit(a)
    srv._admit()
    assert len(srv.active) == 1 and srv.used + srv.pooled - sb <= srv.hbm_budget
    # a pooled state of another shape is freed to make room
    b, other = _spec(512), types.SimpleNamespace(B=256, D=a.hand.dof, s=12, m=5)
    srv = _host_server(hbm_budget=job_bytes(b))
    srv.pool = {("other", 256, 12): [other]}
    srv.pooled = 4 * 256 * (3 * a.hand.dof + 12 * (12 * 5 + 1) + 1)
    srv.submit(b)
    srv._admit()
    assert len(srv.active) == 1 and srv.pool == {} and srv.pooled == 0


def test_eviction_keeps_the_pooled_state_the_job_reuses():
    """The budget only fits the job if other pooled states go: eviction frees
    those and keeps the pooled state of the job's own shape, which the job
    then reuses, so the bytes held stay within the budget."""
    a = _spec(512)
    sb = state_bytes(a)
    mine = types.SimpleNamespace(B=512, D=a.hand.dof, s=12, m=5)
    other = types.SimpleNamespace(B=256, D=a.hand.dof, s=12, m=5)
    ob = 4 * 256 * (3 * a.hand.dof + 12 * (12 * 5 + 1) + 1)
    key = (id(a.hand), 512, 12)
    srv = _host_server(hbm_budget=job_bytes(a) + ob // 2)
    srv.pool = {("other", 256, 12): [other], key: [mine]}  # the other shape first in eviction order
    srv.pooled = sb + ob
    srv.submit(a)
    srv._admit()
    assert len(srv.active) == 1
    assert srv.pool == {key: [mine]} and srv.pooled == sb
    # the job reuses `mine`: held bytes = used + pooled - reused state
    assert srv.used + srv.pooled - sb <= srv.hbm_budget
