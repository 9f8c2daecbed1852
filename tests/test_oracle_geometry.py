"""Pins for the oracle's kinematics, SDF query, tangent basis, energy gradient
and upper-level step (Secs. III, IV-B, IV-C)."""
import json
import math
import os

import numpy as np
import pytest

import bodex_inputs as I
import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


# ----------------------------------------------------------------- FK
def test_fk_zero_pose_is_sum_of_offsets():
    tpl = I.hand_template("hand4")
    H = O.Hand(tpl)
    x = np.zeros((1, tpl.dof))
    c, _, _ = O.fk(H, x)
    # fingers along +y from (x_b, 0.03), thumb along -y from (0, -0.03);
    # links 4 + 3 cm then the tip 2.5 cm further
    L = 0.04 + 0.03 + 0.025
    want = np.array([[-0.02, 0.03 + L, 0], [0.0, 0.03 + L, 0], [0.02, 0.03 + L, 0], [0.0, -0.03 - L, 0]])
    np.testing.assert_allclose(c[0], want, atol=1e-15)


def test_fk_planar_flexion_closed_form():
    tpl = I.hand_template("hand4")
    H = O.Hand(tpl)
    rng = np.random.default_rng(0)
    th = rng.uniform(-1.2, 1.2, size=(5, 3))
    x = np.zeros((5, tpl.dof))
    x[:, 6:9] = th  # first finger
    c, _, _ = O.fk(H, x)
    L = np.array([0.04, 0.03, 0.025])
    cum = np.cumsum(th, axis=1)
    # rotation about +x by a maps +y to (0, cos a, sin a)
    want_y = 0.03 + (L * np.cos(cum)).sum(1)
    want_z = (L * np.sin(cum)).sum(1)
    np.testing.assert_allclose(c[:, 0, 0], -0.02, atol=1e-15)
    np.testing.assert_allclose(c[:, 0, 1], want_y, atol=1e-14)
    np.testing.assert_allclose(c[:, 0, 2], want_z, atol=1e-14)


def test_fk_root_transform_and_orthonormal_frames():
    tpl = I.hand_template("hand5")
    H = O.Hand(tpl)
    obj = I.sphere_object()
    x = I.initial_poses(tpl, obj, 8, seed=5).astype(np.float64)
    fr = O.fk_frames(H, x)
    R = fr[..., :3]
    np.testing.assert_allclose(np.einsum("bjki,bjkl->bjil", R, R), np.broadcast_to(np.eye(3), R.shape), atol=1e-12)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-12)
    # root reading T = Trans(t) Rx Ry Rz, checked on a translated+rotated copy
    x2 = np.zeros((1, tpl.dof))
    x2[0, :6] = [0.1, -0.05, 0.02, 0.3, -0.4, 0.5]
    c0, _, _ = O.fk(H, np.zeros((1, tpl.dof)))
    c2, _, _ = O.fk(H, x2)

    def rot(ax, a):
        c, s = math.cos(a), math.sin(a)
        if ax == 0:
            return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
        if ax == 1:
            return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])
        return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])

    Rr = rot(0, 0.3) @ rot(1, -0.4) @ rot(2, 0.5)
    np.testing.assert_allclose(c2[0], c0[0] @ Rr.T + x2[0, :3], atol=1e-14)


@pytest.mark.parametrize("name", ["hand4", "hand5"])
def test_fk_jacobian_matches_finite_differences(name):
    tpl = I.hand_template(name)
    H = O.Hand(tpl)
    x = I.initial_poses(tpl, I.sphere_object(), 3, seed=9).astype(np.float64)
    c, om, org = O.fk(H, x)
    h = 1e-6
    anc = np.zeros((tpl.n_contacts, tpl.dof), bool)
    anc[:, :6] = True
    for i, j in enumerate(tpl.contact_link):
        while j >= 0:
            anc[i, 6 + j] = True
            j = tpl.parent[j]
    for k in range(tpl.dof):
        xp, xm = x.copy(), x.copy()
        xp[:, k] += h
        xm[:, k] -= h
        fd = (O.fk(H, xp)[0] - O.fk(H, xm)[0]) / (2 * h)
        if k < 3:
            an = np.broadcast_to(om[:, k][:, None, :], fd.shape)
        else:
            an = np.cross(om[:, k][:, None, :], c - org[:, k][:, None, :])
        an = an * anc[None, :, k, None]
        np.testing.assert_allclose(fd, an, atol=1e-8)


# ----------------------------------------------------------------- SDF
def test_sphere_query_exact():
    sph = I.sphere_object(0.04, (0.01, -0.02, 0.005))
    obj = O.Object(sph)
    ctr = sph.center.astype(np.float64)  # the object stores its centre in float32
    rng = np.random.default_rng(1)
    pts = rng.normal(size=(20, 3)) * 0.05
    p, n, phi, deg = O.contact(obj, pts)
    v = pts - ctr
    L = np.linalg.norm(v, axis=1)
    np.testing.assert_allclose(phi, L - 0.04, atol=1e-15)
    np.testing.assert_allclose(p, ctr + 0.04 * v / L[:, None], atol=1e-15)
    np.testing.assert_allclose(n, -v / L[:, None], atol=1e-15)
    assert (deg == 0).all()


def _grid(values_fn, N=16, h=0.01):
    origin = np.full(3, -(N - 1) * h / 2)
    ax = origin[0] + h * np.arange(N)
    zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
    vals = values_fn(np.stack([xx, yy, zz], -1)).astype(np.float32)
    obj = I.GridObject(vals, origin.astype(np.float32), h, [])
    return obj, obj.origin.astype(np.float64)  # the object keeps its origin in float32


def test_grid_reproduces_affine_sdf_exactly():
    nrm = np.array([0.3, -0.5, 0.8])
    nrm /= np.linalg.norm(nrm)
    # a plane SDF sampled at the nodes (node values rounded to float32)
    g, origin = _grid(lambda P: P @ nrm - 0.01)
    obj = O.Object(g)
    vals64 = g.values.astype(np.float64)
    rng = np.random.default_rng(2)
    pts = rng.uniform(-0.06, 0.06, size=(50, 3))
    phi, grad, Hs, cell = O.sdf(obj, pts)
    # trilinear interpolation of the float32 node values, evaluated directly
    u = (pts - origin) / g.h
    c0 = np.clip(np.floor(u).astype(int), 0, g.n - 2)
    t = u - c0
    ref = np.zeros(len(pts))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = (t[:, 0] if dx else 1 - t[:, 0]) * (t[:, 1] if dy else 1 - t[:, 1]) * (t[:, 2] if dz else 1 - t[:, 2])
                ref += w * vals64[c0[:, 2] + dz, c0[:, 1] + dy, c0[:, 0] + dx]
    np.testing.assert_allclose(phi, ref, atol=1e-15)
    # an affine field is reproduced: gradient = normal, zero Hessian
    np.testing.assert_allclose(grad, np.broadcast_to(nrm, grad.shape), atol=2e-6)
    np.testing.assert_allclose(Hs, 0, atol=2e-4)
    np.testing.assert_array_equal(cell, c0)
    p, n, phi2, _ = O.contact(obj, pts)
    np.testing.assert_allclose(n, -np.broadcast_to(nrm, n.shape), atol=2e-6)
    np.testing.assert_allclose(p @ nrm - 0.01, 0, atol=2e-7)


def test_grid_node_values_and_outside_rule():
    g, origin = _grid(lambda P: np.linalg.norm(P, axis=-1) - 0.04, N=12, h=0.01)
    obj = O.Object(g)
    idx = np.array([[0, 0, 0], [3, 5, 7], [11, 11, 11], [11, 0, 4]])
    pts = origin + g.h * idx
    phi, _, _, cell = O.sdf(obj, pts)
    np.testing.assert_allclose(phi, g.values[idx[:, 2], idx[:, 1], idx[:, 0]].astype(np.float64), atol=0)
    assert (cell <= g.n - 2).all() and (cell >= 0).all()
    # outside the box: phi(c) = phi(clamp(c)) + |c - clamp(c)|
    hi = origin + g.h * (g.n - 1)
    out = np.array([[hi[0] + 0.013, 0.001, -0.002], [origin[0] - 0.02, hi[1] + 0.01, 0.003]])
    cl = np.clip(out, origin, hi)
    phi_o, grad_o, _, _ = O.sdf(obj, out)
    phi_c, grad_c, _, _ = O.sdf(obj, cl)
    np.testing.assert_allclose(phi_o, phi_c + np.linalg.norm(out - cl, axis=1), atol=1e-15)
    # gradient along a clamped axis is the unit offset direction
    np.testing.assert_allclose(grad_o[0, 0], 1.0, atol=1e-15)
    np.testing.assert_allclose(grad_o[0, 1:], grad_c[0, 1:], atol=1e-15)


def test_sampled_sphere_within_trilinear_error_bound():
    # h = 2 mm, r = 4 cm: interpolation error <= h^2/8 * sum |d2 phi| ~ 1e-5
    g, _ = _grid(lambda P: np.linalg.norm(P, axis=-1) - 0.04, N=64, h=0.002)
    obj = O.Object(g)
    rng = np.random.default_rng(3)
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pts = d * rng.uniform(0.03, 0.06, size=(200, 1))
    phi, _, _, _ = O.sdf(obj, pts)
    r = np.linalg.norm(pts, axis=1)
    bound = 0.002 ** 2 / 8 * 3 * (2.0 / r) + 1e-7  # |d2 phi| <= 1/r per axis, float32 node rounding
    assert (np.abs(phi - (r - 0.04)) <= bound).all()


def test_sdf_gradient_and_hessian_match_differences():
    g = I.grid_object(seed=7, n=32, h=0.004)
    obj = O.Object(g)
    rng = np.random.default_rng(4)
    pts = rng.uniform(-0.08, 0.08, size=(40, 3))
    phi, grad, Hs, _ = O.sdf(obj, pts)
    h = 1e-7
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        pp, gp, _, cp = O.sdf(obj, pts + e)
        pm, gm, _, cm = O.sdf(obj, pts - e)
        same = (cp == cm).all(1)
        np.testing.assert_allclose(((pp - pm) / (2 * h))[same], grad[same, a], atol=1e-6)
        np.testing.assert_allclose(((gp - gm) / (2 * h))[same], Hs[same][:, :, a], atol=2e-3 * max(1, np.abs(Hs).max()))


def test_grid_gravity_centre_of_sampled_sphere():
    g, _ = _grid(lambda P: np.linalg.norm(P - np.array([0.004, -0.006, 0.002]), axis=-1) - 0.03, N=40, h=0.003)
    obj = O.Object(g)
    np.testing.assert_allclose(obj.gc, [0.004, -0.006, 0.002], atol=1e-3)


# ----------------------------------------------------------------- basis and G
def test_tangent_basis_is_right_handed_orthonormal():
    rng = np.random.default_rng(5)
    n = rng.normal(size=(100, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    d, e = O.basis(n)
    np.testing.assert_allclose((d * d).sum(1), 1, atol=1e-14)
    np.testing.assert_allclose((e * e).sum(1), 1, atol=1e-14)
    np.testing.assert_allclose((d * e).sum(1), 0, atol=1e-14)
    np.testing.assert_allclose(np.cross(d, e), n, atol=1e-14)
    d0, e0 = O.basis(np.array([[0, 0, 1.0], [0, 0, -1.0]]))
    np.testing.assert_allclose(d0, [[1, 0, 0], [1, 0, 0]], atol=0)
    np.testing.assert_allclose(e0, [[0, 1, 0], [0, -1, 0]], atol=0)


def test_grasp_matrix_maps_forces_to_wrenches():
    rng = np.random.default_rng(6)
    p, n = I.random_contacts(5, 3, 8)
    gc = np.array([0.003, -0.001, 0.002])
    G = O.grasp_matrix(p, n, gc)
    d, e = O.basis(n.reshape(-1, 3).astype(np.float64))
    d, e = d.reshape(5, 3, 3), e.reshape(5, 3, 3)
    f = rng.normal(size=(5, 3, 3))
    force = f[..., 0:1] * n + f[..., 1:2] * d + f[..., 2:3] * e
    w = np.einsum("brk,bk->br", G, f.reshape(5, 9))
    np.testing.assert_allclose(w[:, :3], force.sum(1), atol=1e-12)
    np.testing.assert_allclose(w[:, 3:], np.cross(p - gc, force).sum(1), atol=1e-12)


# ----------------------------------------------------------------- energy, gradient, step
@pytest.mark.parametrize("wl", ["tiny", "grid"])
def test_analytic_gradient_matches_central_differences(wl):
    if wl == "tiny":
        hand, obj, x0, T, P, _, _ = I.workload("tiny", batch=12)
    else:
        hand = I.hand_template("hand4")
        obj = I.grid_object(seed=3, n=48, h=0.002)
        x0 = I.initial_poses(hand, obj, 12, seed=4, gap=(0.0, 0.01), flex=0.6)
        T, P = I.wrench_set(12), I.default_params()
    H, Ob = O.Hand(hand), O.Object(obj)
    ev = O.evaluate(H, Ob, x0, T, P)
    gfd = O.grad_fd(H, Ob, x0, T, P, step=1e-6)
    ok = 0
    for b in range(len(x0)):
        # Danskin gradient is defined where y* is unique or the residual is 0;
        # the trilinear Hessian jumps across voxel faces, so skip poses that
        # sit within a few FD steps of one.
        err = np.linalg.norm(ev["grad"][b] - gfd[b]) / max(np.linalg.norm(gfd[b]), 1e-9)
        if err < 1e-5:
            ok += 1
    assert ok >= len(x0) - 1, ok


def test_energy_terms():
    hand, obj, x0, T, P, _, _ = I.workload("tiny", batch=4)
    H, Ob = O.Hand(hand), O.Object(obj)
    ev = O.evaluate(H, Ob, x0, T, P)
    Ed = ((ev["phi"] - hand.contact_radius - P["delta"]) ** 2).sum(1)
    np.testing.assert_allclose(ev["E"], P["w_q"] * ev["Q"].sum(1) + P["w_d"] * Ed, rtol=1e-14)
    # contacts of the analytic sphere lie on it
    np.testing.assert_allclose(np.linalg.norm(ev["p"], axis=-1), 0.04, atol=1e-15)


def test_adam_first_step_and_clamp():
    tpl = I.hand_template("hand4")
    H = O.Hand(tpl)
    P = I.default_params()
    D = tpl.dof
    x = np.zeros((2, D))
    x[1, 6] = tpl.qmax[6] - 1e-4
    g = np.linspace(-3, 3, D)[None].repeat(2, 0)
    g[:, 7] = 0.0
    mm, vv = np.zeros_like(x), np.zeros_like(x)
    x_ref = x.copy()
    O.adam(H, P, x, mm, vv, g, 1)
    lr = np.where(np.arange(D) < 3, P["lr_t"], P["lr_r"])
    # first bias-corrected Adam step: lr * g / (|g| + eps)
    want = np.clip(x_ref - lr * g / (np.abs(g) + P["adam_eps"]), tpl.qmin, tpl.qmax)
    np.testing.assert_allclose(x, want, atol=1e-15)
    assert x[1, 6] <= tpl.qmax[6]


def test_adam_three_steps_golden():
    """Three Adam steps on the gradient sequence g, -g, 2g against the
    hand-derived moments and bias corrections of tests/golden (a step counter
    that never advances, a wrong power of b1 or b2, or a missing bias
    correction changes m-hat or v-hat at step 2 or 3).  One coordinate
    starts half a step below its upper limit: steps 1 and 3 end on the clamp."""
    fx = json.load(open(os.path.join(HERE, "golden", "adam_three_steps.json")))
    tpl = I.hand_template("hand4")
    H = O.Hand(tpl)
    P = I.default_params()
    assert (P["b1"], P["b2"]) == (fx["b1"], fx["b2"])
    D = tpl.dof
    rng = np.random.default_rng(7)
    g = rng.uniform(0.5, 2.0, D) * rng.choice([-1.0, 1.0], D)
    lr = np.where(np.arange(D) < 3, P["lr_t"], P["lr_r"])
    x0 = np.clip(rng.uniform(-0.2, 0.2, D), tpl.qmin, tpl.qmax)
    g[8] = -abs(g[8])  # moves x[8] up at steps 1 and 3
    x0[8] = tpl.qmax[8] - 0.5 * lr[8]
    x, mm, vv = x0[None].copy(), np.zeros((1, D)), np.zeros((1, D))
    want = x0.copy()
    for t in range(3):
        O.adam(H, P, x, mm, vv, (fx["grad_factor"][t] * g)[None], t + 1)
        np.testing.assert_allclose(mm[0], fx["m_coef"][t] * g, rtol=1e-13)
        np.testing.assert_allclose(vv[0], fx["v_coef"][t] * g * g, rtol=1e-13)
        mhat = fx["m_coef"][t] / fx["bias1"][t] * g
        vhat = fx["v_coef"][t] / fx["bias2"][t] * g * g
        want = np.clip(want - lr * mhat / (np.sqrt(vhat) + P["adam_eps"]), tpl.qmin, tpl.qmax)
        np.testing.assert_allclose(x[0], want, rtol=0, atol=1e-14)
    # the clamped coordinate: on the limit after step 1, lr/19 below it after step 2, on it after step 3
    assert x[0, 8] == tpl.qmax[8]


def test_run_decreases_energy_tiny():
    hand, obj, x0, T, P, _, _ = I.workload("tiny", batch=6)
    H, Ob = O.Hand(hand), O.Object(obj)
    E0 = O.evaluate(H, Ob, x0, T, P)["E"]
    x, _, _, _ = O.run(H, Ob, x0, T, P, n_steps=20, grad_mode="analytic")
    E1 = O.evaluate(H, Ob, x, T, P)["E"]
    assert (E1 < E0).all()
    assert (x >= hand.qmin - 1e-12).all() and (x <= hand.qmax + 1e-12).all()


@pytest.mark.parametrize("wl", ["tiny", "grad"])
def test_regularised_energy_gradient_is_exact(wl):
    """With eps |y|^2 the optimum is unique and Q is the regularised optimal
    value, so the envelope-theorem chain is the exact derivative of E: every
    instance agrees with central differences."""
    hand, obj, x0, T, P, _, _ = I.workload(wl, batch=16)
    P = dict(P, eps_reg=1e-3)
    H, Ob = O.Hand(hand), O.Object(obj)
    ev = O.evaluate(H, Ob, x0, T, P)
    gfd = O.grad_fd(H, Ob, x0, T, P, step=1e-6)
    rel = np.linalg.norm(ev["grad"] - gfd, axis=1) / np.linalg.norm(gfd, axis=1)
    assert (rel < 1e-7).all(), rel
