"""Pins for the oracle's cuRobo-style upper-level energies (Sec. IV-B):
hand-object penetration of the collision spheres, self-penetration between
spheres of non-neighbouring links, and the joint-limit penalty (Eq. (4))."""
import math

import numpy as np
import pytest

import bodex_inputs as I
import oracle as O

ONLY = dict(w_q=0.0, w_d=0.0, energy=O.ENERGY_DFC)  # isolate the collision terms (no QPs)


def _params(**kw):
    return dict(I.default_params(), **ONLY, **kw)


def _energy(hand, obj, x, **kw):
    ev = O.evaluate(O.Hand(hand), O.Object(obj), np.atleast_2d(np.asarray(x, np.float64)), I.wrench_set(6),
                    _params(**kw))
    return ev["E"], ev["grad"]


def test_pair_count_of_hand3_is_the_closed_form():
    """hand3: 4 palm spheres, three fingers with 3 + 2 + 2 spheres.  Pairs =
    C(25, 2) minus same-link pairs (6 + 3 (3 + 1 + 1)) minus neighbours per
    finger (palm x link 1: 4 * 3, link 1 x link 2: 3 * 2, link 2 x link 3: 2 * 2)."""
    hand = I.hand_template("hand3")
    assert len(hand.sphere_link) == 25
    same = 6 + 3 * (3 + 1 + 1)
    neigh = 3 * (4 * 3 + 3 * 2 + 2 * 2)
    assert len(O.Hand(hand).pairs()) == math.comb(25, 2) - same - neigh


def test_rest_pose_has_no_self_penetration_and_self_energy_ignores_the_root():
    hand = I.hand_template("hand5")
    obj = I.sphere_object(0.04) if hasattr(I, "sphere_object") else None
    obj = obj or I.workload("tiny", batch=1)[1]
    x = np.zeros(hand.dof)
    E0, _ = _energy(hand, obj, x, w_self=1.0)
    assert E0[0] == 0.0
    # abduct index (joint 0) and middle (joint 4) toward each other by 20 deg:
    # their proximal links cross (bases 2.2 cm apart, 4.5 cm long, spheres of
    # 0.9 cm); E_self > 0 and does not change when the whole hand moves or turns
    xc = x.copy()
    xc[6 + 0] = hand.qmin[6 + 0]
    xc[6 + 4] = hand.qmax[6 + 4]
    E1, _ = _energy(hand, obj, xc, w_self=1.0)
    assert E1[0] > 0
    xm = xc.copy()
    xm[:6] = [0.05, -0.02, 0.3, 0.4, -0.7, 1.1]
    E2, _ = _energy(hand, obj, xm, w_self=1.0)
    np.testing.assert_allclose(E2, E1, rtol=1e-12)


def test_palm_sphere_penetration_is_the_closed_form():
    """Zero joint angles, no rotation: palm sphere k sits at t + local_k.  A
    small sphere object straight below palm sphere 0 (the back of the hand),
    every other sphere outside the activation band, gives
    E = w h(r_0 + eta - (|c_0 - o| - R)) with the hinge h of the reading."""
    hand = I.hand_template("hand3")
    R, eta, w = 0.002, 0.002, 3.0
    l0, r0 = hand.sphere_local[0].astype(np.float64), float(hand.sphere_radius[0])
    H = O.Hand(hand)
    for depth in (0.001, 0.002, 0.005):  # inside the band, at its edge, beyond it
        o = l0 - np.array([0.0, 0.0, R + r0 + eta - depth])
        obj = I.SphereObject(center=o.astype(np.float32), radius=R)
        o = np.asarray(obj.center, np.float64)
        x = np.zeros(hand.dof)
        E, _ = _energy(hand, obj, x, w_pen=w, eta_pen=eta)
        frames = O.fk_frames(H, x[None])[0]
        cs = np.array([frames[L][:, :3] @ hand.sphere_local[s] + frames[L][:, 3] if L >= 0
                       else hand.sphere_local[s].astype(np.float64) for s, L in enumerate(hand.sphere_link)])
        gap = np.linalg.norm(cs - o, axis=1) - R - hand.sphere_radius
        assert (gap[1:] > eta).all(), gap[1:].min()
        p = r0 + eta - (np.linalg.norm(l0 - o) - R)
        h = p * p / (2 * eta) if p <= eta else p - eta / 2
        np.testing.assert_allclose(E[0], w * h, rtol=1e-9)


def test_joint_limit_penalty_closed_form():
    hand = I.hand_template("hand3")
    obj = I.workload("tiny", batch=1)[1]
    x = np.zeros(hand.dof)
    k = 7
    x[k] = float(hand.qmax[k]) - 0.01   # inside the limit, 0.01 from it
    E, g = _energy(hand, obj, x, w_lim=2.0, eta_lim=0.03)  # margin 0.03: excess 0.02
    np.testing.assert_allclose(E[0], 2.0 * 0.02 ** 2, rtol=1e-9)
    np.testing.assert_allclose(g[0, k], 2 * 2.0 * 0.02, rtol=1e-9)
    assert np.count_nonzero(g[0]) == 1
    x[k] = float(hand.qmin[k]) + 0.005
    E, g = _energy(hand, obj, x, w_lim=2.0, eta_lim=0.03)
    np.testing.assert_allclose(E[0], 2.0 * 0.025 ** 2, rtol=1e-9)
    np.testing.assert_allclose(g[0, k], -2 * 2.0 * 0.025, rtol=1e-9)


@pytest.mark.parametrize("kind", ["sphere", "grid"])
def test_collision_gradient_matches_differences(kind):
    if kind == "sphere":
        hand, obj, x, T, P, _, _ = I.workload("tiny", batch=6)
        x = x.astype(np.float64)
        x[:, :3] -= 0.3 * x[:, :3] / np.linalg.norm(x[:, :3], axis=1, keepdims=True) * 0.1  # pull in
    else:
        hand = I.hand_template("hand5")
        obj = I.grid_object(2)
        x = I.initial_poses(hand, obj, 6, seed=41, gap=(-0.02, 0.0), flex=1.0).astype(np.float64)
    rng = np.random.default_rng(5)
    x[:, 6:] = np.clip(x[:, 6:] + rng.uniform(-0.6, 0.6, size=x[:, 6:].shape), hand.qmin[6:], hand.qmax[6:])
    prm = _params(w_pen=2.0, w_self=5.0, w_lim=1.0, eta_pen=0.005, eta_lim=0.2)
    H, Ob = O.Hand(hand), O.Object(obj)
    T6 = I.wrench_set(6)
    ev = O.evaluate(H, Ob, x, T6, prm)
    on = ev["E"] > 0
    assert on.sum() >= 3
    gf = O.grad_fd(H, Ob, x, T6, prm, step=1e-7)
    rel = np.linalg.norm(ev["grad"] - gf, axis=1)[on] / np.linalg.norm(gf, axis=1)[on]
    assert (rel < 1e-5).all(), rel


def test_collision_terms_add_to_the_grasp_energy():
    hand, obj, x, T, P, _, _ = I.workload("tiny", batch=4)
    x = x.astype(np.float64)
    H, Ob = O.Hand(hand), O.Object(obj)
    base = O.evaluate(H, Ob, x, T, P)["E"]
    coll = O.evaluate(H, Ob, x, T, dict(P, w_q=0.0, w_d=0.0, energy=O.ENERGY_DFC, w_self=1.0, w_pen=1.0))["E"]
    both = O.evaluate(H, Ob, x, T, dict(P, w_self=1.0, w_pen=1.0))["E"]
    np.testing.assert_allclose(both, base + coll, rtol=1e-12)
