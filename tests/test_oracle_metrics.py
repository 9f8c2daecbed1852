"""Pins for the oracle's Contact Distance Consistency metric (Sec. V-B):
cdc = max_i d_i - min_i d_i over the fingers, d_i the signed distance of
fingertip i (smallest phi over its surface samples; phi(c_i) - alpha for a
hand without samples)."""
import dataclasses

import numpy as np

import bodex_inputs as I
import oracle as O


def _sphere_case(batch=8, seed=21):
    hand, obj, x0, _, _, _, _ = I.workload("tiny", batch=batch)
    rng = np.random.default_rng(seed)
    x = x0.astype(np.float64)
    x[:, 6:] += rng.uniform(-0.2, 0.2, size=x[:, 6:].shape)
    return hand, obj, x


def test_fingertip_distance_is_the_closest_sample_on_a_sphere():
    """Brute force over the samples with the closed-form sphere distance
    |p - o| - r, through the (separately pinned) link frames."""
    hand, obj, x = _sphere_case()
    H, Ob = O.Hand(hand), O.Object(obj)
    r = O.contact_metrics(H, Ob, x)
    frames = O.fk_frames(H, x)
    tips = hand.tip_samples.astype(np.float64)
    o, rad = np.asarray(obj.center, np.float64), float(obj.radius)
    want = np.zeros((len(x), hand.n_contacts))
    for b in range(len(x)):
        for i, link in enumerate(hand.contact_link):
            F = frames[b, link]
            pts = tips[i] @ F[:, :3].T + F[:, 3]
            want[b, i] = (np.linalg.norm(pts - o, axis=1) - rad).min()
    np.testing.assert_allclose(r["d"], want, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["cdc"], want.max(1) - want.min(1), rtol=0, atol=1e-12)


def test_hand_without_samples_uses_the_coarse_sphere():
    hand, obj, x = _sphere_case()
    bare = dataclasses.replace(hand, tip_samples=None)
    H, Ob = O.Hand(bare), O.Object(obj)
    r = O.contact_metrics(H, Ob, x)
    c = O.fk(H, x)[0]
    want = np.linalg.norm(c - np.asarray(obj.center, np.float64), axis=-1) - obj.radius - hand.contact_radius
    np.testing.assert_allclose(r["d"], want, rtol=0, atol=1e-12)


def test_sampled_distance_brackets_the_exact_fingertip_sphere_distance():
    """Samples lie on the fingertip sphere (radius alpha around c_i), so for a
    sphere object phi(c_i) - alpha <= d_i <= phi(c_i) - alpha cos(theta), with
    theta the largest angle between the object direction and its nearest
    sample direction (bounded by the sample spacing)."""
    hand, obj, x = _sphere_case(batch=16, seed=3)
    H, Ob = O.Hand(hand), O.Object(obj)
    r = O.contact_metrics(H, Ob, x)
    c = O.fk(H, x)[0]
    phi_c = np.linalg.norm(c - np.asarray(obj.center, np.float64), axis=-1) - obj.radius
    a = hand.contact_radius
    assert (r["d"] >= phi_c - a - 1e-12).all()
    # 32 Fibonacci points on the sphere: every direction is within 40 degrees of one
    assert (r["d"] <= phi_c - a * np.cos(np.radians(40.0)) + 1e-12).all()


def test_metric_is_invariant_to_moving_hand_and_object_together():
    hand, obj, x = _sphere_case()
    shift = np.array([0.013, -0.021, 0.007])
    moved = dataclasses.replace(obj, center=(np.asarray(obj.center, np.float64) + shift).astype(np.float32))
    x2 = x.copy()
    x2[:, :3] += np.asarray(moved.center, np.float64) - np.asarray(obj.center, np.float64)
    r1 = O.contact_metrics(O.Hand(hand), O.Object(obj), x)
    r2 = O.contact_metrics(O.Hand(hand), O.Object(moved), x2)
    np.testing.assert_allclose(r2["d"], r1["d"], atol=1e-12)
    np.testing.assert_allclose(r2["cdc"], r1["cdc"], atol=1e-12)
    assert (r1["cdc"] >= 0).all()


def test_grid_metric_matches_the_sampled_sdf():
    """On the grid object, d_i equals the smallest oracle SDF value over the
    transformed samples (the SDF itself is pinned in test_oracle_geometry)."""
    hand = I.hand_template("hand5")
    obj = I.grid_object(2)
    x = I.initial_poses(hand, obj, 6, seed=12, gap=(-0.01, 0.005), flex=0.8).astype(np.float64)
    H, Ob = O.Hand(hand), O.Object(obj)
    r = O.contact_metrics(H, Ob, x)
    frames = O.fk_frames(H, x)
    tips = hand.tip_samples.astype(np.float64)
    for b in range(len(x)):
        for i, link in enumerate(hand.contact_link):
            F = frames[b, link]
            phi = O.sdf(Ob, tips[i] @ F[:, :3].T + F[:, 3])[0]
            assert abs(phi.min() - r["d"][b, i]) < 1e-12
