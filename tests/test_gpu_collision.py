"""cuRobo-style constraint energies (Sec. IV-B: joint limits, hand-object and
hand-hand penetration on collision spheres) on the GPU vs the FP64 oracle.
FP32 sums of squared penetrations: E relative 1e-4; gradient relative 1e-3
(off voxel faces for the grid)."""
import dataclasses

import numpy as np
import pytest

from gpu_helpers import I, O, cuda, host, torch

import paper_2412_16490_gb300 as bx

pytestmark = pytest.mark.gpu

COLL = dict(w_pen=2.0, w_self=5.0, w_lim=1.0, eta_pen=0.005, eta_lim=0.2)


def _off_faces(obj, c, tol=1e-3):
    if obj.kind == "sphere":
        return np.ones(c.shape[:-1], bool)
    lo = np.asarray(obj.origin, np.float64)
    hi = lo + obj.h * (obj.n - 1)
    u = (c - lo) / obj.h
    inside = (c >= lo) & (c <= hi)
    ok_in = np.abs(u - np.round(u)) > tol
    ok_out = np.minimum(np.abs(c - lo), np.abs(c - hi)) > tol * obj.h
    return np.where(inside, ok_in, ok_out).all(-1)


def _root(xb):
    """T_root = Trans(t) Rx Ry Rz (the pose reading of the hand descriptor)."""
    def rot(axis, a):
        c, s = np.cos(a), np.sin(a)
        i, j = [(1, 2), (2, 0), (0, 1)][axis]
        R = np.eye(3)
        R[i, i], R[i, j], R[j, i], R[j, j] = c, -s, s, c
        return R
    return rot(0, xb[3]) @ rot(1, xb[4]) @ rot(2, xb[5]), xb[:3]


def _sphere_centres(hand, H, x):
    frames = O.fk_frames(H, x)
    out = np.zeros((len(x), len(hand.sphere_link), 3))
    for b in range(len(x)):
        R0, t0 = _root(x[b])
        for k, L in enumerate(hand.sphere_link):
            F = frames[b, L] if L >= 0 else np.concatenate([R0, t0[:, None]], 1)
            out[b, k] = F[:, :3] @ hand.sphere_local[k] + F[:, 3]
    return out


def _case(kind, B, seed=5):
    """Poses with penetration, self-contact and joints near their limits."""
    if kind == "tiny":
        hand, obj, x, T, P, _, _ = I.workload("tiny", batch=B)
        x = x.astype(np.float64)
        x[:, :3] *= 0.7  # the palm moves toward the sphere at the origin
    else:
        hand, obj, _, T, P, _, _ = I.workload("paper", batch=1)
        x = I.initial_poses(hand, obj, B, seed=41, gap=(-0.02, 0.0), flex=1.0).astype(np.float64)
    rng = np.random.default_rng(seed)
    x[:, 6:] = np.clip(x[:, 6:] + rng.uniform(-1.2, 1.2, size=x[:, 6:].shape), hand.qmin[6:], hand.qmax[6:])
    return hand, obj, x.astype(np.float32), T, P


@pytest.mark.parametrize("kind,B", [("tiny", 37), ("paper", 48)])
@pytest.mark.parametrize("energy", ["dfc_only_collision", "qp_plus_collision"])
def test_collision_energy_and_gradient_match_oracle(kind, B, energy):
    hand, obj, x0, T, P = _case(kind, B)
    if energy == "dfc_only_collision":
        Pr = dict(P, w_q=0.0, w_d=0.0, energy=bx.ENERGY_DFC, **COLL)
        sp = bx.step_params(Pr)
    else:
        Pr = dict(P, eps_reg=1e-3, **COLL)
        sp = bx.step_params(Pr, qp=bx.qp_params(eps_abs=1e-6, eps_reg=1e-3, max_iter=20000, check_every=10))
    H, Ob = bx.Hand(hand), bx.Object(obj)
    out = bx.bodex_energy_grad(H, Ob, cuda(x0), cuda(T), sp)
    Po = dict(Pr, energy=O.ENERGY_DFC if energy == "dfc_only_collision" else O.ENERGY_QP)
    Ho = O.Hand(hand)
    ev = O.evaluate(Ho, O.Object(obj), x0.astype(np.float64), T, Po)
    st = host(out["status"])
    ok = (st & bx.ST_NOT_CONVERGED) == 0
    if obj.kind != "sphere":
        cs = _sphere_centres(hand, Ho, x0.astype(np.float64))
        ok &= _off_faces(obj, ev["c"]).all(-1) & _off_faces(obj, cs).all(-1)
    assert ok.sum() >= B // 3
    E = host(out["E"])
    if energy == "dfc_only_collision":
        assert (ev["E"][ok] > 0).mean() > 0.5
    np.testing.assert_allclose(E[ok], ev["E"][ok], rtol=1e-4, atol=1e-6)
    g, gref = host(out["dEdx"]), ev["grad"]
    rel = np.linalg.norm(g - gref, axis=1) / np.maximum(np.linalg.norm(gref, axis=1), 1e-3)
    assert (rel[ok] <= 1e-3).all(), rel[ok].max()


def test_collision_terms_are_off_at_zero_weight():
    hand, obj, x0, T, P = _case("tiny", 16)
    H, Ob = bx.Hand(hand), bx.Object(obj)
    base = bx.bodex_energy_grad(H, Ob, cuda(x0), cuda(T), bx.step_params(P))
    zero = bx.bodex_energy_grad(H, Ob, cuda(x0), cuda(T), bx.step_params(dict(P, w_pen=0.0, w_self=0.0, w_lim=0.0)))
    assert torch.equal(base["E"], zero["E"]) and torch.equal(base["dEdx"], zero["dEdx"])


def test_limit_energy_without_spheres():
    hand, obj, x0, T, P = _case("tiny", 16)
    bare = dataclasses.replace(hand, sphere_link=None, sphere_local=None, sphere_radius=None)
    Pr = dict(P, w_q=0.0, w_d=0.0, energy=bx.ENERGY_DFC, w_lim=3.0, eta_lim=0.3)
    out = bx.bodex_energy_grad(bx.Hand(bare), bx.Object(obj), cuda(x0), cuda(T), bx.step_params(Pr))
    ev = O.evaluate(O.Hand(bare), O.Object(obj), x0.astype(np.float64), T, dict(Pr, energy=O.ENERGY_DFC))
    np.testing.assert_allclose(host(out["E"]), ev["E"], rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(host(out["dEdx"]), ev["grad"], rtol=1e-5, atol=1e-7)


def test_collision_step_is_adam_and_lowers_the_collision_energy():
    hand, obj, x0, T, P = _case("tiny", 32)
    Pr = dict(P, w_q=0.0, w_d=0.0, energy=bx.ENERGY_DFC, **COLL)
    H, Ob = bx.Hand(hand), bx.Object(obj)
    sp = bx.step_params(Pr)
    x = cuda(x0)
    ev0 = bx.bodex_energy_grad(H, Ob, x, cuda(T), sp)
    g = host(ev0["dEdx"])
    st = bx.State(H, 32, T.shape[0])
    st.set_pose(x)
    E = torch.empty(32, device="cuda")
    bx.bodex_step(H, Ob, st, cuda(T), 1, sp, E_last=E)
    lr = np.where(np.arange(hand.dof) < 3, P["lr_t"], P["lr_r"])
    want = np.clip(x0 - lr * g / (np.abs(g) + P["adam_eps"]), hand.qmin, hand.qmax)
    np.testing.assert_allclose(host(st.pose()), want, atol=2e-6)
    bx.bodex_step(H, Ob, st, cuda(T), 100, sp, E_last=E)
    E0 = host(ev0["E"])
    on = E0 > 0
    assert np.median(host(E)[on] / E0[on]) < 0.5


def test_collision_in_a_mixed_launch_matches_single_launches():
    """bodex_step_multi with the collision energies on: each job's result
    equals its own bodex_step launch (bitwise)."""
    Pr = dict(I.default_params(), **COLL)
    sp = bx.step_params(Pr, qp=bx.qp_params(max_iter=20))
    jobs, singles = [], []
    for name, B, seed in (("hand3", 40, 1), ("hand5", 24, 2)):
        hand = I.hand_template(name)
        obj = I.grid_object(seed, n=48)
        x0 = I.initial_poses(hand, obj, B, seed=seed)
        T = cuda(I.wrench_set(12))
        H, Ob = bx.Hand(hand), bx.Object(obj)
        a, b = bx.State(H, B, 12), bx.State(H, B, 12)
        a.set_pose(cuda(x0))
        b.set_pose(cuda(x0))
        Ea, Eb = torch.empty(B, device="cuda"), torch.empty(B, device="cuda")
        jobs.append(dict(hand=H, obj=Ob, state=a, T=T, n_steps=10, E_last=Ea))
        bx.bodex_step(H, Ob, b, T, 10, sp, E_last=Eb)
        singles.append((a, b, Ea, Eb))
    bx.bodex_step_multi(jobs, sp)
    for a, b, Ea, Eb in singles:
        assert torch.equal(a.pose(), b.pose())
        assert torch.equal(Ea, Eb)
