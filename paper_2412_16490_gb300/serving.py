"""Continuous-batching synthesis server.

Jobs (an object, a hand template, a batch of initial poses, a step count)
arrive at any time.  `Server` keeps every admitted job's pose, Adam moments
and ADMM warm starts resident on the device and, each tick, advances all
active jobs together in ONE mixed-template launch (`bodex_step_multi`):
jobs that arrive while others run join at the next tick, as soon as device
memory (an HBM budget) and a job slot allow; finished jobs leave, their
results are read back and their memory is freed.  A grasp's result does not
depend on which other jobs shared its launches.

`PlainServer` is the baseline: one job at a time, first come first served,
one kernel launch per upper iteration.

Both record, per job, latency = completion time - arrival time.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import Hand, Object, State, bodex_step, bodex_step_multi, bodex_step_tile, step_params
from ._binding import BODEX_MAX_JOBS

CTAS_PER_SM = 4   # resident thread blocks of the fused step kernel per SM (register bound)


@dataclass
class JobSpec:
    """One synthesis request."""
    hand: object                 # a bodex_inputs.HandTemplate
    obj: object                  # a SphereObject or GridObject
    x0: np.ndarray               # [B, 6+n] float32 initial poses (host)
    T: np.ndarray                # [s, 6] desired wrenches
    n_steps: int = 200
    arrival: float = 0.0         # seconds after the server's start (replays)
    tag: object = None


@dataclass
class JobResult:
    x: np.ndarray                # [B, 6+n] final poses
    E: np.ndarray                # [B] energy at the last evaluated pose
    arrival: float
    start: float
    finish: float
    tag: object = None
    res: np.ndarray | None = None  # [B] largest QP residual (ADMM) or Frank-Wolfe gap (exact) of the last step

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


@dataclass
class _Active:
    jid: int
    spec: JobSpec
    hand: Hand
    obj: Object
    state: State
    T: object
    E: object
    remaining: int
    start: float
    nbytes: int


def state_bytes(spec: JobSpec) -> int:
    """Device bytes of the job's optimiser state: pose, Adam moments, ADMM
    warm starts and residual."""
    B, D = spec.x0.shape
    m, s = spec.hand.n_contacts, spec.T.shape[0]
    return 4 * B * (3 * D + s * (3 * m + 9 * m + 1) + 1)


def job_bytes(spec: JobSpec) -> int:
    """Device bytes a job holds while admitted: its state, energy and
    wrenches (objects are shared, see object_bytes)."""
    return state_bytes(spec) + 4 * (spec.x0.shape[0] + 6 * spec.T.shape[0])


def _state_key(spec: JobSpec):
    return id(spec.hand), spec.x0.shape[0], spec.T.shape[0]


def object_bytes(obj) -> int:
    return 0 if obj.kind == "sphere" else 4 * int(obj.values.size)


class _Base:
    def __init__(self, params: dict | None = None, qp=None, grasps_per_cta: int = 0):
        self.params = step_params(params, qp=qp, grasps_per_cta=grasps_per_cta)
        self._hands: dict = {}
        self._objects: dict = {}  # id(obj) -> [Object, users]
        self._lock = threading.Lock()
        self._waiting: deque = deque()
        self._next_id = 0
        self.results: dict = {}
        self.t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def _hand(self, tpl) -> Hand:
        h = self._hands.get(id(tpl))
        if h is None:
            h = self._hands[id(tpl)] = Hand(tpl)
        return h

    def _object(self, o) -> Object:
        ent = self._objects.get(id(o))
        if ent is None:
            ent = self._objects[id(o)] = [Object(o), 0]
        ent[1] += 1
        return ent[0]

    def _release_object(self, o) -> int:
        """Drops one user of the object; frees it (returns its bytes) when unused."""
        ent = self._objects[id(o)]
        ent[1] -= 1
        if ent[1] == 0:
            del self._objects[id(o)]
            return object_bytes(o)
        return 0

    def submit(self, spec: JobSpec, arrival: float | None = None) -> int:
        """Queue a job; returns its id.  Thread-safe."""
        with self._lock:
            jid = self._next_id
            self._next_id += 1
            spec.arrival = self.now() if arrival is None else arrival
            self._waiting.append((jid, spec))
        return jid

    def poll(self) -> list:
        """Ids of the finished jobs."""
        return list(self.results)

    def result(self, jid: int) -> JobResult:
        return self.results[jid]

    def _new_state(self, spec, hand) -> State:
        return State(hand, spec.x0.shape[0], spec.T.shape[0])

    def _open(self, jid, spec):
        import torch
        hand = self._hand(spec.hand)
        obj = self._object(spec.obj)
        st = self._new_state(spec, hand)
        x = torch.as_tensor(np.ascontiguousarray(spec.x0, np.float32)).pin_memory().cuda(non_blocking=True)
        st.set_pose(x)
        T = torch.as_tensor(np.ascontiguousarray(spec.T, np.float32)).cuda()
        E = torch.empty(spec.x0.shape[0], dtype=torch.float32, device="cuda")
        return _Active(jid, spec, hand, obj, st, T, E, spec.n_steps, self.now(), job_bytes(spec))

    def _close(self, a: _Active):
        x = a.state.pose().cpu().numpy()
        E = a.E.cpu().numpy()
        res = a.state.residual().cpu().numpy()
        self.results[a.jid] = JobResult(x, E, a.spec.arrival, a.start, self.now(), a.spec.tag, res)
        return self._release_object(a.spec.obj)

    def replay(self, specs, realtime: bool = True, idle_sleep: float = 2e-4):
        """Serve `specs` arriving at their `arrival` times (seconds after the
        start of the replay); returns {id: JobResult}."""
        order = sorted(range(len(specs)), key=lambda k: specs[k].arrival)
        self.t0 = time.perf_counter()
        nxt = 0
        ids = {}
        while nxt < len(order) or self.busy():
            now = self.now()
            while nxt < len(order) and (not realtime or specs[order[nxt]].arrival <= now):
                k = order[nxt]
                ids[k] = self.submit(specs[k], arrival=specs[k].arrival if realtime else now)
                nxt += 1
            if self.busy():
                self.tick()
            elif nxt < len(order):
                time.sleep(min(idle_sleep, max(0.0, specs[order[nxt]].arrival - self.now())))
        return {k: self.results[j] for k, j in ids.items()}


class Server(_Base):
    """Continuous batching over one mixed-template launch per tick.

    Ticks are enqueued without waiting for the device: each tick advances
    every active job by up to `steps_per_tick` upper iterations in one
    launch.  A job whose last step is in a tick has its result copied to
    pinned host memory behind that launch and an event recorded; it is
    reported finished (and its memory freed) when the event completes.  At
    most `max_inflight` ticks are queued on the device, so a job that
    arrives joins within that many ticks.

    Finished jobs return their optimiser state to a pool keyed by (hand,
    batch, wrenches) and the next job of that shape reuses it: freeing device
    memory synchronises the whole device, which would stall the queued
    ticks.  Pooled states count against the HBM budget; when a job does not
    fit, pooled states are freed first."""

    def __init__(self, params: dict | None = None, qp=None, steps_per_tick: int = 10, hbm_budget: int | None = None,
                 max_jobs: int = BODEX_MAX_JOBS, grasps_per_cta: int = 0, max_inflight: int = 2,
                 max_waves: float | None = 1.0):
        super().__init__(params, qp, grasps_per_cta)
        import torch
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info()
            hbm_budget = int(free * 0.8)
        self.hbm_budget = int(hbm_budget)
        # thread blocks resident at once: a launch beyond one wave slows every
        # job in it, so admission stops there (None: no limit)
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        self.cta_budget = None if max_waves is None else max(1, int(max_waves * sms * CTAS_PER_SM))
        self.ctas = 0
        self.steps_per_tick = int(steps_per_tick)
        self.max_jobs = min(int(max_jobs), BODEX_MAX_JOBS)
        self.max_inflight = max(1, int(max_inflight))
        self.active: list = []      # jobs with steps left
        self.finishing: list = []   # (job, event, pinned x, E, residual): last tick enqueued
        self.inflight: deque = deque()
        self.used = 0
        self.pool: dict = {}        # _state_key -> [State]
        self.pooled = 0             # bytes held by pooled states
        self.launches = 0
        self.peak_active = 0
        self.peak_used = 0

    def busy(self) -> bool:
        return bool(self.active or self._waiting or self.finishing)

    def _job_ctas(self, spec) -> int:
        gpb = bodex_step_tile(spec.hand.n_contacts, spec.T.shape[0], self.params.grasps_per_cta)
        return -(-spec.x0.shape[0] // gpb)

    def _new_state(self, spec, hand) -> State:
        lst = self.pool.get(_state_key(spec))
        if lst:
            self.pooled -= state_bytes(spec)
            return lst.pop()
        return super()._new_state(spec, hand)

    def _evict_pool(self, need: int, keep=None):
        """Frees pooled states until `need` more bytes fit the budget, never
        the pool of shape `keep` (the state the admitted job will reuse)."""
        for key in list(self.pool):
            if key == keep:
                continue
            lst = self.pool[key]
            while lst and self.used + self.pooled + need > self.hbm_budget:
                st = lst.pop()
                self.pooled -= 4 * st.B * (3 * st.D + st.s * (12 * st.m + 1) + 1)
                del st
            if not lst:
                del self.pool[key]

    def _admit(self):
        while self._waiting and len(self.active) + len(self.finishing) < self.max_jobs:
            jid, spec = self._waiting[0]
            nb = job_bytes(spec) + (0 if id(spec.obj) in self._objects else object_bytes(spec.obj))
            # a pooled state of the same shape is reused: its bytes are already held
            reuse = state_bytes(spec) if self.pool.get(_state_key(spec)) else 0
            if self.used + self.pooled + nb - reuse > self.hbm_budget:
                self._evict_pool(nb - reuse, keep=_state_key(spec))
            if self.used + self.pooled + nb - reuse > self.hbm_budget:
                if not self.active and not self.finishing and nb > self.hbm_budget:
                    raise MemoryError(f"job {jid} needs {nb} bytes, over the HBM budget {self.hbm_budget}")
                break  # wait for memory to free up
            nc = self._job_ctas(spec)
            if self.cta_budget is not None and self.active and self.ctas + nc > self.cta_budget:
                break  # wait for a wave's worth of thread blocks to free up
            with self._lock:
                self._waiting.popleft()
            self.active.append(self._open(jid, spec))
            self.active[-1].nbytes = job_bytes(spec)
            self.used += nb
            self.ctas += nc
            self.peak_active = max(self.peak_active, len(self.active) + len(self.finishing))
            self.peak_used = max(self.peak_used, self.used + self.pooled)

    def _reap(self, block: bool = False):
        keep = []
        for a, ev, xh, Eh, rh in self.finishing:
            if block:
                ev.synchronize()
            if block or ev.query():
                self.results[a.jid] = JobResult(xh.numpy().copy(), Eh.numpy().copy(), a.spec.arrival, a.start,
                                                self.now(), a.spec.tag, rh.numpy().copy())
                self.used -= a.nbytes + self._release_object(a.spec.obj)
                self.pool.setdefault(_state_key(a.spec), []).append(a.state)
                self.pooled += state_bytes(a.spec)
                a.state = None
            else:
                keep.append((a, ev, xh, Eh, rh))
        self.finishing = keep
        while self.inflight and self.inflight[0].query():
            self.inflight.popleft()

    def tick(self):
        """Reap finished jobs, admit what fits, enqueue one launch for every
        active job (at most steps_per_tick iterations each)."""
        import torch
        self._reap()
        self._admit()
        if not self.active:
            if self.finishing:
                time.sleep(5e-5)
            return
        while len(self.inflight) >= self.max_inflight:
            self.inflight.popleft().synchronize()
        table = []
        for a in self.active:
            n = min(self.steps_per_tick, a.remaining)
            table.append(dict(hand=a.hand, obj=a.obj, state=a.state, T=a.T, n_steps=n, E_last=a.E))
            a.remaining -= n
        bodex_step_multi(table, self.params)
        self.launches += 1
        keep = []
        for a in self.active:
            if a.remaining == 0:
                self.ctas -= self._job_ctas(a.spec)
                xh = torch.empty((a.spec.x0.shape[0], a.hand.D), dtype=torch.float32).pin_memory()
                Eh = torch.empty(a.spec.x0.shape[0], dtype=torch.float32).pin_memory()
                rh = torch.empty(a.spec.x0.shape[0], dtype=torch.float32).pin_memory()
                xh.copy_(a.state.pose(), non_blocking=True)
                Eh.copy_(a.E, non_blocking=True)
                rh.copy_(a.state.residual(), non_blocking=True)
                ev = torch.cuda.Event()
                ev.record()
                self.finishing.append((a, ev, xh, Eh, rh))
            else:
                keep.append(a)
        self.active = keep
        ev = torch.cuda.Event()
        ev.record()
        self.inflight.append(ev)


class PlainServer(_Base):
    """Baseline: one job at a time (FIFO), one launch per upper iteration."""

    def __init__(self, params: dict | None = None, qp=None, grasps_per_cta: int = 0):
        super().__init__(params, qp, grasps_per_cta)
        self.launches = 0

    def busy(self) -> bool:
        return bool(self._waiting)

    def tick(self):
        import torch
        with self._lock:
            jid, spec = self._waiting.popleft()
        a = self._open(jid, spec)
        for _ in range(spec.n_steps):
            bodex_step(a.hand, a.obj, a.state, a.T, 1, self.params, E_last=a.E)
            self.launches += 1
        torch.cuda.current_stream().synchronize()
        self._close(a)


def latency_stats(results: dict) -> dict:
    lat = np.array([r.latency for r in results.values()])
    grasps = sum(r.x.shape[0] for r in results.values())
    span = max(r.finish for r in results.values()) - min(r.arrival for r in results.values())
    out = dict(p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
               mean_s=float(lat.mean()), jobs=len(lat), grasps=int(grasps), span_s=float(span),
               grasps_per_s=float(grasps / span) if span > 0 else None)
    if all(r.res is not None for r in results.values()):
        res = np.concatenate([r.res for r in results.values()])
        out["frac_grasps_all_qps_le_1e-5"] = float((res <= 1e-5).mean())
    return out


@dataclass
class PoissonWorkload:
    """Poisson arrivals of synthesis jobs (seeded): grids of 32-128 nodes per
    axis, one of the three hand templates, 256-4096 grasps, 200 steps."""
    n_jobs: int = 300
    rate: float = 20.0
    seed: int = 5
    n_steps: int = 200
    grasp_choices: tuple = (256, 512, 1024, 2048, 4096)
    grid_choices: tuple = (32, 48, 64, 96, 128)
    templates: tuple = ("hand3", "hand4x4", "hand5")
    specs: list = field(default_factory=list)

    def build(self):
        import bodex_inputs as I
        rng = np.random.default_rng(self.seed)
        grids = {n: I.grid_object(self.seed * 10 + k, n=n, h=0.128 / (n - 1))
                 for k, n in enumerate(self.grid_choices)}
        hands = {t: I.hand_template(t) for t in self.templates}
        pools = {}
        t = 0.0
        T = I.wrench_set(12)
        self.specs = []
        for j in range(self.n_jobs):
            t += rng.exponential(1.0 / self.rate)
            n = self.grid_choices[int(rng.integers(len(self.grid_choices)))]
            tn = self.templates[int(rng.integers(len(self.templates)))]
            B = self.grasp_choices[int(rng.integers(len(self.grasp_choices)))]
            key = (tn, n)
            if key not in pools:
                pools[key] = I.initial_poses(hands[tn], grids[n], max(self.grasp_choices),
                                             seed=self.seed * 7919 + len(pools))
            off = int(rng.integers(0, max(self.grasp_choices) - B + 1))
            self.specs.append(JobSpec(hands[tn], grids[n], pools[key][off:off + B], T, self.n_steps, t,
                                      tag=dict(job=j, template=tn, grid=n, grasps=B)))
        return self.specs
