"""GB300-native BODex coarse-stage hot path (arXiv 2412.16490).

Python face of the C ABI in ``include/bodex.h``.  Functions carry the
ABI's names and only marshal arguments: torch CUDA tensors supply device
memory, ``torch.cuda.current_stream()`` the stream.  All arithmetic runs in
the CUDA library ``libbodex.so`` built from ``csrc/``; if that library is
missing or cannot load, importing the compute functions raises -- there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _binding as _b
from ._binding import BodexError, CONE_ELLIPTIC, CONE_PYRAMID, ENERGY_DFC, ENERGY_QP, ST_DEGENERATE_NORMAL, ST_NONFINITE, ST_NOT_CONVERGED, ST_POLISHED, QP_ADMM, QP_EXACT  # noqa: F401

__all__ = [
    "load", "Hand", "Object", "State", "qp_params", "step_params",
    "bodex_hand_create", "bodex_object_create", "bodex_state_create",
    "bodex_fk_contacts", "bodex_qp_solve_batch", "bodex_energy_grad", "bodex_energy_adjoint", "bodex_step", "bodex_step_multi", "bodex_refine",
    "bodex_contact_metrics", "bodex_squeeze_pose", "synthesize",
    "bodex_sync", "bodex_version", "bodex_step_tile", "BodexError",
]


def load():
    """Build (if needed) and load the CUDA library; returns the ctypes handle."""
    return _b.load()


def _torch():
    import torch
    return torch


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("bodex arrays must be CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("bodex arrays must be contiguous")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _np(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ---------------------------------------------------------------- parameters
def qp_params(mu=0.5, beta=1.0, gamma=0.5, rho=0.1, sigma=1e-6, alpha=1.6, eps_abs=0.0, eps_reg=0.0,
              max_iter=50, check_every=10, warm=0, strict=0, cone=0, adaptive_rho=0,
              polish=0, solver=0) -> _b.bodex_qp_params:
    """ADMM/QP parameters (struct bodex_qp_params); cone: CONE_PYRAMID or
    CONE_ELLIPTIC; adaptive_rho: residual-balancing rho in solves with a
    residual target (eps_abs > 0); polish: the exact FP64 solve after ADMM
    in bodex_qp_solve_batch; solver: QP_ADMM or QP_EXACT (the float32
    minimum-norm-point method; max_iter caps its oracle calls)."""
    return _b.bodex_qp_params(mu, beta, gamma, rho, sigma, alpha, eps_abs, eps_reg, int(max_iter),
                              int(check_every), int(warm), int(strict), int(cone), int(adaptive_rho), int(polish),
                              int(solver))


def step_params(params: dict | None = None, qp: _b.bodex_qp_params | None = None,
                grasps_per_cta: int = 0, work_pulling: int = 0) -> _b.bodex_step_params:
    """Upper-level parameters (struct bodex_step_params) from a dict with keys
    lr_t, lr_r, b1, b2, adam_eps, w_q, w_d, delta, energy (ENERGY_QP or
    ENERGY_DFC), the collision energies w_pen, w_self, w_lim, eta_pen, eta_lim
    (off at weight 0), and mu, beta, gamma, eps_reg used when `qp` is not
    given."""
    p = dict(lr_t=2e-3, lr_r=2e-2, b1=0.9, b2=0.999, adam_eps=1e-8, w_q=1.0, w_d=1000.0, delta=0.01,
             mu=0.5, beta=1.0, gamma=0.5, eps_reg=0.0, energy=_b.ENERGY_QP, w_pen=0.0, w_self=0.0, w_lim=0.0,
             eta_pen=0.005, eta_lim=0.0)
    if params:
        p.update({k: v for k, v in params.items() if k in p})
    if qp is None:
        qp = qp_params(mu=p["mu"], beta=p["beta"], gamma=p["gamma"], eps_reg=p["eps_reg"])
    return _b.bodex_step_params(p["lr_t"], p["lr_r"], p["b1"], p["b2"], p["adam_eps"],
                                _b.bodex_energy_params(p["w_q"], p["w_d"], p["delta"], int(p["energy"]), p["w_pen"],
                                                       p["w_self"], p["w_lim"], p["eta_pen"], p["eta_lim"]), qp,
                                int(grasps_per_cta), int(work_pulling))


# ---------------------------------------------------------------- handles
class Hand:
    """Device copy of a hand template (bodex_hand_create)."""

    def __init__(self, tpl):
        L = load()
        self.tpl = tpl
        self.n, self.m = int(tpl.n_joints), int(tpl.n_contacts)
        self.D = 6 + self.n
        keep = dict(parent=_np(tpl.parent, np.int32), offset=_np(tpl.offset, np.float32),
                    axis=_np(tpl.axis, np.float32), qmin=_np(tpl.qmin, np.float32),
                    qmax=_np(tpl.qmax, np.float32), clink=_np(tpl.contact_link, np.int32),
                    clocal=_np(tpl.contact_local, np.float32))
        tips = getattr(tpl, "tip_samples", None)
        S = 0 if tips is None else int(tips.shape[1])
        keep["tips"] = _np(tips, np.float32) if tips is not None else None
        sl = getattr(tpl, "sphere_link", None)
        K = 0 if sl is None else int(len(sl))
        keep["sl"] = _np(sl, np.int32) if K else None
        keep["sp"] = _np(tpl.sphere_local, np.float32) if K else None
        keep["sr"] = _np(tpl.sphere_radius, np.float32) if K else None
        fp = lambda a: a.ctypes.data_as(_b.c_float_p) if a is not None else None
        ip = lambda a: a.ctypes.data_as(_b.c_int_p) if a is not None else None
        desc = _b.bodex_hand_desc(self.n, self.m, ip(keep["parent"]), fp(keep["offset"]), fp(keep["axis"]),
                                  fp(keep["qmin"]), fp(keep["qmax"]), ip(keep["clink"]), fp(keep["clocal"]),
                                  float(tpl.contact_radius), S, fp(keep["tips"]), K, ip(keep["sl"]),
                                  fp(keep["sp"]), fp(keep["sr"]))
        self.K = K
        h = C.c_void_p()
        _b.check(L.bodex_hand_create(C.byref(desc), C.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) and _b._lib is not None:
            _b._lib.bodex_hand_destroy(self._h)
            self._h = None


class Object:
    """Device copy of an object: analytic sphere or node-sampled SDF grid."""

    def __init__(self, obj, stream=None):
        L = load()
        self.obj = obj
        if obj.kind == "sphere":
            c = _np(obj.center, np.float32)
            desc = _b.bodex_object_desc(0, (C.c_float * 3)(*c), float(obj.radius), 0, 0.0,
                                        (C.c_float * 3)(0, 0, 0), None)
            self._vals = None
        else:
            self._vals = _np(obj.values, np.float32)
            org = _np(obj.origin, np.float32)
            desc = _b.bodex_object_desc(1, (C.c_float * 3)(0, 0, 0), 0.0, int(self._vals.shape[0]),
                                        float(obj.h), (C.c_float * 3)(*org),
                                        self._vals.ctypes.data_as(_b.c_float_p))
        o = C.c_void_p()
        _b.check(L.bodex_object_create(C.byref(desc), _stream(stream), C.byref(o)))
        self._o = o
        gc = (C.c_float * 3)()
        _b.check(L.bodex_object_gravity_centre(o, gc))
        self.gc = np.array(gc[:], np.float32)

    @property
    def handle(self):
        return self._o

    def __del__(self):
        if getattr(self, "_o", None) and _b._lib is not None:
            _b._lib.bodex_object_destroy(self._o)
            self._o = None


class State:
    """Optimiser state for B grasps and s wrenches (bodex_state_create)."""

    def __init__(self, hand: Hand, B: int, s: int):
        L = load()
        st = C.c_void_p()
        _b.check(L.bodex_state_create(hand.handle, int(B), int(s), C.byref(st)))
        self._s = st
        self.B, self.s, self.D, self.m = int(B), int(s), hand.D, hand.m

    @property
    def handle(self):
        return self._s

    def set_pose(self, x, stream=None):
        _b.check(load().bodex_state_set_pose(self._s, _ptr(x), _stream(stream)))

    def pose(self, stream=None):
        torch = _torch()
        x = torch.empty((self.B, self.D), dtype=torch.float32, device="cuda")
        _b.check(load().bodex_state_get_pose(self._s, _ptr(x), _stream(stream)))
        return x

    def residual(self, stream=None):
        """Per-grasp max ADMM residual at the last step of the last launch [B]."""
        torch = _torch()
        r = torch.empty(self.B, dtype=torch.float32, device="cuda")
        _b.check(load().bodex_state_get_residual(self._s, _ptr(r), _stream(stream)))
        return r

    def adam(self, stream=None):
        torch = _torch()
        m = torch.empty((self.B, self.D), dtype=torch.float32, device="cuda")
        v = torch.empty_like(m)
        t = C.c_int()
        _b.check(load().bodex_state_get_adam(self._s, _ptr(m), _ptr(v), C.byref(t), _stream(stream)))
        return m, v, t.value

    def __del__(self):
        if getattr(self, "_s", None) and _b._lib is not None:
            _b._lib.bodex_state_destroy(self._s)
            self._s = None


def bodex_hand_create(tpl) -> Hand:
    return Hand(tpl)


def bodex_object_create(obj, stream=None) -> Object:
    return Object(obj, stream)


def bodex_state_create(hand: Hand, B: int, s: int) -> State:
    return State(hand, B, s)


# ---------------------------------------------------------------- calls
def bodex_fk_contacts(hand: Hand, obj: Object, x, stream=None):
    """FK + nearest-point query + G for poses x [B,D] (CUDA float32)."""
    torch = _torch()
    B, m = int(x.shape[0]), hand.m
    f = lambda *s: torch.empty(s, dtype=torch.float32, device=x.device)
    out = dict(c=f(B, m, 3), p=f(B, m, 3), n=f(B, m, 3), phi=f(B, m), G=f(B, 6, 3 * m),
               cell=torch.empty((B, m, 3), dtype=torch.int32, device=x.device),
               status=torch.empty((B,), dtype=torch.int32, device=x.device))
    _b.check(load().bodex_fk_contacts(hand.handle, obj.handle, _ptr(x), B, _ptr(out["c"]), _ptr(out["p"]),
                                      _ptr(out["n"]), _ptr(out["phi"]), _ptr(out["G"]), _ptr(out["cell"]),
                                      _ptr(out["status"]), _stream(stream)))
    return out


def bodex_qp_solve_batch(G, T, params: _b.bodex_qp_params, y=None, z=None, lam=None, stream=None):
    """Batched QPs for G [B,6,3m] and wrenches T [s,6].  y/z/lam are the warm
    start (used when params.warm) and are overwritten with the result."""
    torch = _torch()
    B, nv = int(G.shape[0]), int(G.shape[2])
    m, s = nv // 3, int(T.shape[0])
    nc = 4 * m + 1 if params.cone == _b.CONE_ELLIPTIC else 9 * m + 1
    dev = G.device
    f = lambda *sh: torch.zeros(sh, dtype=torch.float32, device=dev)
    y = f(B, s, nv) if y is None else y
    z = f(B, s, nc) if z is None else z
    lam = f(B, s, nc) if lam is None else lam
    Q = f(B, s)
    iters = torch.zeros((B, s), dtype=torch.int32, device=dev)
    status = torch.zeros((B, s), dtype=torch.int32, device=dev)
    res = f(B, s, 2)
    _b.check(load().bodex_qp_solve_batch(_ptr(G), B, m, _ptr(T), s, C.byref(params), _ptr(y), _ptr(z),
                                         _ptr(lam), _ptr(Q), _ptr(iters), _ptr(status), _ptr(res),
                                         _stream(stream)))
    return dict(y=y, z=z, lam=lam, Q=Q, iters=iters, status=status, res=res)


def bodex_energy_grad(hand: Hand, obj: Object, x, T, params: _b.bodex_step_params, warm: State | None = None,
                      stream=None):
    """E [B], dE/dx [B,D], Q [B,s], y [B,s,3m], status [B] at poses x."""
    torch = _torch()
    B, s = int(x.shape[0]), int(T.shape[0])
    dev = x.device
    out = dict(E=torch.empty(B, dtype=torch.float32, device=dev),
               dEdx=torch.empty((B, hand.D), dtype=torch.float32, device=dev),
               Q=torch.empty((B, s), dtype=torch.float32, device=dev),
               y=torch.empty((B, s, 3 * hand.m), dtype=torch.float32, device=dev),
               status=torch.empty(B, dtype=torch.int32, device=dev))
    _b.check(load().bodex_energy_grad(hand.handle, obj.handle, _ptr(x), B, _ptr(T), s, C.byref(params),
                                      warm.handle if warm is not None else None, _ptr(out["E"]),
                                      _ptr(out["dEdx"]), _ptr(out["Q"]), _ptr(out["y"]), _ptr(out["status"]),
                                      _stream(stream)))
    return out


def bodex_energy_adjoint(hand: Hand, obj: Object, x, T, params: _b.bodex_step_params, y, stream=None):
    """dE/dx [B,D] and E [B] at poses x for given forces y [B,s,3m] (no QP solve)."""
    torch = _torch()
    B, s = int(x.shape[0]), int(T.shape[0])
    dev = x.device
    out = dict(E=torch.empty(B, dtype=torch.float32, device=dev),
               dEdx=torch.empty((B, hand.D), dtype=torch.float32, device=dev),
               status=torch.empty(B, dtype=torch.int32, device=dev))
    _b.check(load().bodex_energy_adjoint(hand.handle, obj.handle, _ptr(x), B, _ptr(T), s, C.byref(params), _ptr(y),
                                         _ptr(out["E"]), _ptr(out["dEdx"]), _ptr(out["status"]), _stream(stream)))
    return out


def bodex_step(hand: Hand, obj: Object, state: State, T, n_steps: int, params: _b.bodex_step_params,
               E_last=None, status=None, stream=None):
    """n_steps fused upper iterations on `state`; returns (E_last, status)."""
    _b.check(load().bodex_step(hand.handle, obj.handle, state.handle, _ptr(T), int(T.shape[0]), int(n_steps),
                               C.byref(params), _ptr(E_last), _ptr(status), _stream(stream)))
    return E_last, status


def bodex_refine(hand: Hand, obj: Object, state: State, p_coarse, n_steps: int, delta: float, w_qp: float,
                 params: _b.bodex_step_params, E_last=None, kstar=None, status=None, stream=None):
    """n_steps refinement iterations (fine stage: delta = 0.01, final: 0)."""
    _b.check(load().bodex_refine(hand.handle, obj.handle, state.handle, _ptr(p_coarse), int(n_steps), float(delta),
                                 float(w_qp), C.byref(params), _ptr(E_last), _ptr(kstar), _ptr(status),
                                 _stream(stream)))
    return E_last, kstar, status


def bodex_contact_metrics(hand: Hand, obj: Object, x, stream=None):
    """Signed fingertip distances d [B,m] and Contact Distance Consistency
    cdc [B] = max_i d_i - min_i d_i (Sec. V-B), in metres."""
    torch = _torch()
    B = int(x.shape[0])
    d = torch.empty((B, hand.m), dtype=torch.float32, device=x.device)
    cdc = torch.empty(B, dtype=torch.float32, device=x.device)
    _b.check(load().bodex_contact_metrics(hand.handle, obj.handle, _ptr(x), B, _ptr(d), _ptr(cdc), _stream(stream)))
    return dict(d=d, cdc=cdc)


def bodex_squeeze_pose(x, x_p, stream=None):
    """Squeeze pose x_s = 2 x - x_p (Sec. IV-D) for poses x, x_p [B,D]."""
    torch = _torch()
    B, D = int(x.shape[0]), int(x.shape[1])
    x_s = torch.empty((B, D), dtype=torch.float32, device=x.device)
    _b.check(load().bodex_squeeze_pose(_ptr(x), _ptr(x_p), B, D, _ptr(x_s), _stream(stream)))
    return x_s


def synthesize(hand: Hand, obj: Object, x0, T, params: _b.bodex_step_params, coarse_steps=300, fine_steps=100,
               final_steps=100, margin=0.01, w_qp=1000.0, stream=None):
    """The three-stage schedule (Sec. IV-D; 300 / 100 / 100 iterations):
    coarse steps with the QP energy, then fine steps (pre-grasp x_p, margin)
    and final steps (grasp x), and the squeeze pose x_s = 2 x - x_p.
    Returns dict x_p, x, x_s, E and the grasp's fingertip distances d and
    Contact Distance Consistency cdc (Sec. V-B)."""
    torch = _torch()
    B = int(x0.shape[0])
    st = State(hand, B, int(T.shape[0]))
    st.set_pose(x0, stream)
    E = torch.empty(B, dtype=torch.float32, device=x0.device)
    bodex_step(hand, obj, st, T, coarse_steps, params, E_last=E, stream=stream)
    pc = bodex_fk_contacts(hand, obj, st.pose(stream), stream)["p"]
    bodex_refine(hand, obj, st, pc, fine_steps, margin, w_qp, params, E_last=E, stream=stream)
    xp = st.pose(stream)
    bodex_refine(hand, obj, st, pc, final_steps, 0.0, w_qp, params, E_last=E, stream=stream)
    x = st.pose(stream)
    met = bodex_contact_metrics(hand, obj, x, stream)
    return dict(x_p=xp, x=x, x_s=bodex_squeeze_pose(x, xp, stream), E=E, d=met["d"], cdc=met["cdc"])


def bodex_step_multi(jobs, params: _b.bodex_step_params, stream=None):
    """One launch for several jobs.  jobs: iterable of dicts with keys hand,
    obj, state, T, n_steps and optionally E_last, status (CUDA tensors)."""
    jobs = list(jobs)
    arr = (_b.bodex_job * max(1, len(jobs)))()
    for k, j in enumerate(jobs):
        T = j["T"]
        arr[k] = _b.bodex_job(j["hand"].handle, j["obj"].handle, j["state"].handle, _ptr(T), int(T.shape[0]),
                              int(j["n_steps"]), _ptr(j.get("E_last")), _ptr(j.get("status")))
    _b.check(load().bodex_step_multi(arr, len(jobs), C.byref(params), _stream(stream)))


def bodex_sync(stream=None):
    _b.check(load().bodex_sync(_stream(stream)))


def bodex_version() -> str:
    return load().bodex_version().decode()


def bodex_step_tile(m: int, s: int, requested: int = 0) -> int:
    """Grasps per thread block the fused step kernel uses for m contacts and
    s wrenches (`requested` = grasps_per_cta, 0 for the default).  Host-only."""
    out = C.c_int(0)
    _b.check(load().bodex_step_tile(int(m), int(s), int(requested), C.byref(out)))
    return out.value
