"""FP64 CPU oracle for the BODex coarse-stage inner loop -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never does; the two
share no code.  The arithmetic lives in ``bodex_oracle.cpp`` (plain C++17,
double precision); this module compiles it with g++ on first use and wraps
its C interface with ctypes.

Every function here is a thin marshalling layer.  See the C++ file for the
paper passages each routine follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bodex_oracle.cpp")
_LIB = os.path.join(_HERE, "libbodex_oracle.so")
_lock = threading.Lock()
_lib = None

PARAM_KEYS = ("mu", "beta", "gamma", "w_q", "w_d", "delta", "eps_reg",
              "lr_t", "lr_r", "b1", "b2", "adam_eps", "energy",
              "w_pen", "w_self", "w_lim", "eta_pen", "eta_lim", "cone", "cone_facets")
ENERGY_QP, ENERGY_DFC = 0, 1
CONE_PYRAMID, CONE_ELLIPTIC = 0, 1
_PARAM_DEFAULTS = {"energy": ENERGY_QP, "w_pen": 0.0, "w_self": 0.0, "w_lim": 0.0, "eta_pen": 0.005,
                   "eta_lim": 0.0, "cone": CONE_PYRAMID, "cone_facets": 512}


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, -O2) if it is missing or stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _sig(_lib)
    return _lib


_d = C.POINTER(C.c_double)
_f = C.POINTER(C.c_float)
_i = C.POINTER(C.c_int32)
_v = C.c_void_p


def _sig(L):
    L.orc_hand_new.restype = _v
    L.orc_hand_new.argtypes = [C.c_int, C.c_int, _i, _f, _f, _f, _f, _i, _f, C.c_double, C.c_int, _f,
                               C.c_int, _i, _f, _f]
    L.orc_hand_pairs.restype = C.c_int
    L.orc_hand_pairs.argtypes = [_v, _i]
    L.orc_hand_free.argtypes = [_v]
    L.orc_object_sphere.restype = _v
    L.orc_object_sphere.argtypes = [C.c_double] * 4
    L.orc_object_grid.restype = _v
    L.orc_object_grid.argtypes = [C.c_int, C.c_double, _f, _f]
    L.orc_object_free.argtypes = [_v]
    L.orc_object_gc.argtypes = [_v, _d]
    L.orc_fk.argtypes = [_v, _d, C.c_int, _d, _d, _d]
    L.orc_fk_frames.argtypes = [_v, _d, C.c_int, _d]
    L.orc_sdf.argtypes = [_v, _d, C.c_int, _d, _d, _d, _i]
    L.orc_contact.argtypes = [_v, _d, C.c_int, _d, _d, _d, _i]
    L.orc_basis.argtypes = [_d, C.c_int, _d, _d]
    L.orc_grasp_matrix.argtypes = [_d, _d, C.c_int, C.c_int, _d, _d]
    L.orc_qp_solve.argtypes = [_d, C.c_int, C.c_int, _d, C.c_int] + [C.c_double] * 4 + [C.c_int, _d, _d, _d, _i, _i, _d, _i]
    L.orc_qp_bruteforce.argtypes = [_d, C.c_int, C.c_int, _d, C.c_int] + [C.c_double] * 4 + [C.c_int, _d, _d]
    L.orc_evaluate.argtypes = [_v, _v, _d, C.c_int, _d, _d, C.c_int, C.c_int,
                               _d, _d, _d, _d, _d, _i, _d, _d, _d, _i, _d, _i]
    L.orc_grad_fd.argtypes = [_v, _v, _d, C.c_int, _d, _d, C.c_int, C.c_double, C.c_int, _d]
    L.orc_adam.argtypes = [_v, _d, _d, _d, _d, _d, C.c_int, C.c_int]
    L.orc_run.argtypes = [_v, _v, _d, _d, _d, C.c_int, C.c_int, C.c_int, _d, _d, C.c_int,
                          C.c_int, C.c_double, C.c_int, _d]
    L.orc_refine_eval.argtypes = [_v, _v, _d, C.c_int, _d, C.c_double, C.c_double, C.c_double, C.c_int,
                                  _d, _d, _i, _d]
    L.orc_refine_run.argtypes = [_v, _v, _d, _d, _d, C.c_int, _d, C.c_int, C.c_int, C.c_double, C.c_double,
                                 _d, C.c_int, _d]
    L.orc_contact_metrics.argtypes = [_v, _v, _d, C.c_int, C.c_int, _d, _d]
    L.orc_qp_soc.argtypes = [_d, C.c_int, C.c_int, _d, C.c_int] + [C.c_double] * 4 + [C.c_int, C.c_int, _d, _d, _d,
                                                                                        _d, _i, _d]


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


class Hand:
    """Oracle copy of a hand template (values promoted to float64)."""

    def __init__(self, tpl):
        L = _load()
        self.tpl = tpl
        self.n, self.m = tpl.n_joints, tpl.n_contacts
        self.D = 6 + self.n
        keep = [np.ascontiguousarray(tpl.parent, np.int32), _f32(tpl.offset), _f32(tpl.axis),
                _f32(tpl.qmin), _f32(tpl.qmax), np.ascontiguousarray(tpl.contact_link, np.int32),
                _f32(tpl.contact_local)]
        tips = tpl.tip_samples
        S = 0 if tips is None else int(tips.shape[1])
        tips = _f32(tips) if tips is not None else None
        sl = getattr(tpl, "sphere_link", None)
        K = 0 if sl is None else int(len(sl))
        sph = [np.ascontiguousarray(sl, np.int32), _f32(tpl.sphere_local), _f32(tpl.sphere_radius)] if K else [None] * 3
        self.K = K
        self._h = L.orc_hand_new(self.n, self.m, _p(keep[0], _i), _p(keep[1], _f), _p(keep[2], _f),
                                 _p(keep[3], _f), _p(keep[4], _f), _p(keep[5], _i), _p(keep[6], _f),
                                 float(tpl.contact_radius), S, _p(tips, _f), K, _p(sph[0], _i), _p(sph[1], _f),
                                 _p(sph[2], _f))

    def pairs(self) -> np.ndarray:
        """Self-collision sphere pairs [P, 2] (spheres on non-neighbouring links)."""
        n = _load().orc_hand_pairs(self._h, None)
        out = np.zeros((n, 2), np.int32)
        _load().orc_hand_pairs(self._h, _p(out, _i))
        return out

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_hand_free(self._h)
            self._h = None


class Object:
    """Oracle copy of an object: analytic sphere or node-sampled grid."""

    def __init__(self, obj):
        L = _load()
        self.obj = obj
        if obj.kind == "sphere":
            c = np.asarray(obj.center, np.float64)
            self._o = L.orc_object_sphere(float(c[0]), float(c[1]), float(c[2]), float(obj.radius))
        else:
            vals = _f32(obj.values)
            org = _f32(obj.origin)
            self._o = L.orc_object_grid(int(vals.shape[0]), float(obj.h), _p(org, _f), _p(vals, _f))
        gc = np.zeros(3)
        L.orc_object_gc(self._o, _p(gc, _d))
        self.gc = gc

    def __del__(self):
        if getattr(self, "_o", None) and _lib is not None:
            _lib.orc_object_free(self._o)
            self._o = None


def params_array(params: dict) -> np.ndarray:
    return np.array([float(params.get(k, _PARAM_DEFAULTS.get(k))) for k in PARAM_KEYS], np.float64)


def fk(hand: Hand, x):
    x = _f64(x).reshape(-1, hand.D)
    B = x.shape[0]
    c = np.zeros((B, hand.m, 3))
    om = np.zeros((B, hand.D, 3))
    org = np.zeros((B, hand.D, 3))
    _load().orc_fk(hand._h, _p(x, _d), B, _p(c, _d), _p(om, _d), _p(org, _d))
    return c, om, org


def fk_frames(hand: Hand, x):
    x = _f64(x).reshape(-1, hand.D)
    fr = np.zeros((x.shape[0], hand.n, 3, 4))
    _load().orc_fk_frames(hand._h, _p(x, _d), x.shape[0], _p(fr, _d))
    return fr


def sdf(obj: Object, pts):
    pts = _f64(pts).reshape(-1, 3)
    K = pts.shape[0]
    phi, g, H = np.zeros(K), np.zeros((K, 3)), np.zeros((K, 3, 3))
    cell = np.zeros((K, 3), np.int32)
    _load().orc_sdf(obj._o, _p(pts, _d), K, _p(phi, _d), _p(g, _d), _p(H, _d), _p(cell, _i))
    return phi, g, H, cell


def contact(obj: Object, pts):
    pts = _f64(pts).reshape(-1, 3)
    K = pts.shape[0]
    p, n, phi = np.zeros((K, 3)), np.zeros((K, 3)), np.zeros(K)
    deg = np.zeros(K, np.int32)
    _load().orc_contact(obj._o, _p(pts, _d), K, _p(p, _d), _p(n, _d), _p(phi, _d), _p(deg, _i))
    return p, n, phi, deg


def basis(n):
    n = _f64(n).reshape(-1, 3)
    d, e = np.zeros_like(n), np.zeros_like(n)
    _load().orc_basis(_p(n, _d), n.shape[0], _p(d, _d), _p(e, _d))
    return d, e


def grasp_matrix(p, n, gc=(0.0, 0.0, 0.0)):
    p = _f64(p)
    n = _f64(n)
    B, m = p.shape[0], p.shape[1]
    G = np.zeros((B, 6, 3 * m))
    gcv = _f64(gc)
    _load().orc_grasp_matrix(_p(p, _d), _p(n, _d), B, m, _p(gcv, _d), _p(G, _d))
    return G


def qp_solve(G, T, mu=0.5, beta=1.0, gamma=0.5, eps_reg=0.0, threads=None, want_lam=False):
    """Exact QP (active set).  Returns dict y [B,s,3m], Q, kkt, unique, status, iters (, lam)."""
    G = _f64(G)
    T = _f64(T)
    B, nv = G.shape[0], G.shape[2]
    m, s = nv // 3, T.shape[0]
    y = np.zeros((B, s, nv))
    Q, kkt = np.zeros((B, s)), np.zeros((B, s))
    uq, st, it = (np.zeros((B, s), np.int32) for _ in range(3))
    lam = np.zeros((B, s, 10 * m + 1)) if want_lam else None
    _load().orc_qp_solve(_p(G, _d), B, m, _p(T, _d), s, mu, beta, gamma, eps_reg,
                         threads or default_threads(), _p(y, _d), _p(Q, _d), _p(kkt, _d),
                         _p(uq, _i), _p(st, _i), _p(lam, _d), _p(it, _i))
    out = dict(y=y, Q=Q, kkt=kkt, unique=uq, status=st, iters=it)
    if want_lam:
        out["lam"] = lam
    return out


def qp_soc(G, T, mu=0.5, beta=1.0, gamma=0.5, eps_reg=0.0, K=256, threads=None):
    """Elliptic friction cone (the unlinearised contact model), bracketed by
    exact QPs over the K-facet pyramids inscribed in and circumscribed about
    the cone: Q_out <= Q* <= Q_in.  Returns dict y [B,s,3m] (the inscribed
    optimum, feasible for the cone), Q_in, Q_out, kkt, status, lam
    [B,s,4m+1] (rows: per contact f_n, the cone rows (mu f_n, f_d, f_e); then
    the sum row)."""
    G = _f64(G)
    T = _f64(T)
    B, nv = G.shape[0], G.shape[2]
    m, s = nv // 3, T.shape[0]
    y = np.zeros((B, s, nv))
    Qi, Qo, kkt = np.zeros((B, s)), np.zeros((B, s)), np.zeros((B, s))
    st = np.zeros((B, s), np.int32)
    lam = np.zeros((B, s, 4 * m + 1))
    _load().orc_qp_soc(_p(G, _d), B, m, _p(T, _d), s, mu, beta, gamma, eps_reg, int(K), threads or default_threads(),
                       _p(y, _d), _p(Qi, _d), _p(Qo, _d), _p(kkt, _d), _p(st, _i), _p(lam, _d))
    return dict(y=y, Q_in=Qi, Q_out=Qo, kkt=kkt, status=st, lam=lam)


def qp_bruteforce(G, T, mu=0.5, beta=1.0, gamma=0.5, eps_reg=0.0, threads=None):
    G = _f64(G)
    T = _f64(T)
    B, nv = G.shape[0], G.shape[2]
    m, s = nv // 3, T.shape[0]
    if m > 3:
        raise ValueError("brute force is limited to m <= 3")
    Q = np.zeros((B, s))
    y = np.zeros((B, s, nv))
    _load().orc_qp_bruteforce(_p(G, _d), B, m, _p(T, _d), s, mu, beta, gamma, eps_reg,
                              threads or default_threads(), _p(Q, _d), _p(y, _d))
    return Q, y


def evaluate(hand: Hand, obj: Object, x, T, params, threads=None):
    """E and every intermediate at B poses (analytic gradient included)."""
    x = _f64(x).reshape(-1, hand.D)
    T = _f64(T)
    B, m, s, nv = x.shape[0], hand.m, T.shape[0], 3 * hand.m
    out = dict(E=np.zeros(B), c=np.zeros((B, m, 3)), p=np.zeros((B, m, 3)), n=np.zeros((B, m, 3)),
               phi=np.zeros((B, m)), cell=np.zeros((B, m, 3), np.int32), G=np.zeros((B, 6, nv)),
               Q=np.zeros((B, s)), y=np.zeros((B, s, nv)), unique=np.zeros((B, s), np.int32),
               grad=np.zeros((B, hand.D)), status=np.zeros(B, np.int32))
    pa = params_array(params)
    _load().orc_evaluate(hand._h, obj._o, _p(x, _d), B, _p(pa, _d), _p(T, _d), s,
                         threads or default_threads(),
                         *[_p(out[k], _i if out[k].dtype == np.int32 else _d)
                           for k in ("E", "c", "p", "n", "phi", "cell", "G", "Q", "y", "unique", "grad", "status")])
    return out


def grad_fd(hand: Hand, obj: Object, x, T, params, step=1e-6, threads=None):
    x = _f64(x).reshape(-1, hand.D)
    T = _f64(T)
    g = np.zeros_like(x)
    pa = params_array(params)
    _load().orc_grad_fd(hand._h, obj._o, _p(x, _d), x.shape[0], _p(pa, _d), _p(T, _d), T.shape[0],
                        step, threads or default_threads(), _p(g, _d))
    return g


def adam(hand: Hand, params, x, mm, vv, grad, t):
    """In-place Adam + clamp on float64 arrays x, mm, vv [B,D]."""
    pa = params_array(params)
    for a in (x, mm, vv):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _f64(grad)
    _load().orc_adam(hand._h, _p(pa, _d), _p(x, _d), _p(mm, _d), _p(vv, _d), _p(g, _d), x.shape[0], t)


def run(hand: Hand, obj: Object, x0, T, params, n_steps, grad_mode="fd", t0=0, mm=None, vv=None,
        fd_step=1e-6, threads=None):
    """The coarse-stage loop for B grasps.  Returns (x, mm, vv, E_last)."""
    x = _f64(x0).reshape(-1, hand.D).copy()
    B = x.shape[0]
    mm = np.zeros_like(x) if mm is None else _f64(mm).copy()
    vv = np.zeros_like(x) if vv is None else _f64(vv).copy()
    E = np.zeros(B)
    T = _f64(T)
    pa = params_array(params)
    _load().orc_run(hand._h, obj._o, _p(x, _d), _p(mm, _d), _p(vv, _d), B, n_steps, t0, _p(pa, _d),
                    _p(T, _d), T.shape[0], 0 if grad_mode == "fd" else 1, fd_step,
                    threads or default_threads(), _p(E, _d))
    return x, mm, vv, E


def refine_eval(hand: Hand, obj: Object, x, p_coarse, delta, w_d, w_qp, threads=None):
    """Refinement energy (fine/final stages) at B poses: E, grad, kstar, gap."""
    x = _f64(x).reshape(-1, hand.D)
    B = x.shape[0]
    pc = _f64(p_coarse).reshape(B, hand.m, 3)
    E, g = np.zeros(B), np.zeros((B, hand.D))
    k = np.zeros((B, hand.m), np.int32)
    gap = np.zeros((B, hand.m))
    _load().orc_refine_eval(hand._h, obj._o, _p(x, _d), B, _p(pc, _d), float(delta), float(w_d), float(w_qp),
                            threads or default_threads(), _p(E, _d), _p(g, _d), _p(k, _i), _p(gap, _d))
    return dict(E=E, grad=g, kstar=k, gap=gap)


def contact_metrics(hand: Hand, obj: Object, x, threads=None):
    """Signed fingertip distances d [B,m] and Contact Distance Consistency
    cdc [B] = max_i d_i - min_i d_i (Sec. V-B), in metres."""
    x = _f64(x).reshape(-1, hand.D)
    B = x.shape[0]
    d, cdc = np.zeros((B, hand.m)), np.zeros(B)
    _load().orc_contact_metrics(hand._h, obj._o, _p(x, _d), B, threads or default_threads(), _p(d, _d), _p(cdc, _d))
    return dict(d=d, cdc=cdc)


def refine_run(hand: Hand, obj: Object, x, mm, vv, p_coarse, n_steps, t0, delta, w_qp, params, threads=None):
    """n_steps refinement iterations with Adam; returns (x, mm, vv, E_last)."""
    x = _f64(x).reshape(-1, hand.D).copy()
    mm, vv = _f64(mm).copy(), _f64(vv).copy()
    B = x.shape[0]
    pc = _f64(p_coarse).reshape(B, hand.m, 3)
    E = np.zeros(B)
    pa = params_array(params)
    _load().orc_refine_run(hand._h, obj._o, _p(x, _d), _p(mm, _d), _p(vv, _d), B, _p(pc, _d), int(n_steps), int(t0),
                           float(delta), float(w_qp), _p(pa, _d), threads or default_threads(), _p(E, _d))
    return x, mm, vv, E
