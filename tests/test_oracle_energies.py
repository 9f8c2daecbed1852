"""Pins for the switchable comparison energies (Sec. V-C): the DFC
force-closure energy of Liu et al. 2021 (frictionless, equal unit normal
forces: E_Q = |sum_i [n_i; p_i x n_i]|^2) and the QP baseline (our QP energy
with beta = 0)."""
import numpy as np
import pytest

import bodex_inputs as I
import oracle as O


def _sphere(batch=12):
    hand, obj, x0, T, P, _, _ = I.workload("tiny", batch=batch)
    return hand, obj, x0.astype(np.float64), T, P


def test_dfc_energy_on_a_sphere_is_the_closed_form():
    """On a sphere the inward normals are radial and the contact points are
    relative to the centre, so every torque p_i x n_i vanishes and
    E = w_Q |sum_i (o - c_i)/|o - c_i||^2 + w_d sum_i (|c_i - o| - r - alpha - delta)^2."""
    hand, obj, x, T, P = _sphere()
    Pd = dict(P, energy=O.ENERGY_DFC)
    ev = O.evaluate(O.Hand(hand), O.Object(obj), x, T, Pd)
    c = O.fk(O.Hand(hand), x)[0]
    o = np.asarray(obj.center, np.float64)
    v = o - c
    L = np.linalg.norm(v, axis=-1)
    n_sum = (v / L[..., None]).sum(1)
    Ed = ((L - obj.radius - hand.contact_radius - P["delta"]) ** 2).sum(1)
    want = P["w_q"] * (n_sum ** 2).sum(1) + P["w_d"] * Ed
    np.testing.assert_allclose(ev["E"], want, rtol=1e-12, atol=1e-15)
    assert (ev["Q"] == 0).all()  # no lower-level QPs under DFC


def test_dfc_vanishes_for_opposed_contacts():
    """Two pairs of diametrically opposed contacts on a sphere are force
    closure in the DFC sense: the normals cancel and there is no torque."""
    n = np.array([[1.0, 0, 0], [-1.0, 0, 0], [0, 0.6, 0.8], [0, -0.6, -0.8]])
    p = -0.04 * n  # points on a 4 cm sphere around the origin, inward normals
    G = O.grasp_matrix(p[None], n[None])[0]
    w = G[:, 0::3].sum(1)  # G u
    np.testing.assert_allclose(w, 0.0, atol=1e-15)


@pytest.mark.parametrize("kind", ["sphere", "grid"])
def test_dfc_gradient_matches_differences(kind):
    if kind == "sphere":
        hand, obj, x, T, P = _sphere(6)
    else:
        hand = I.hand_template("hand5")
        obj = I.grid_object(2)
        x = I.initial_poses(hand, obj, 6, seed=31, gap=(0.0, 0.01), flex=0.6).astype(np.float64)
        T, P = I.wrench_set(12), I.default_params()
    Pd = dict(P, energy=O.ENERGY_DFC)
    H, Ob = O.Hand(hand), O.Object(obj)
    ga = O.evaluate(H, Ob, x, T, Pd)["grad"]
    gf = O.grad_fd(H, Ob, x, T, Pd, step=1e-6)
    rel = np.linalg.norm(ga - gf, axis=1) / np.linalg.norm(gf, axis=1)
    assert (rel < 1e-5).all(), rel


def test_qp_baseline_is_beta_zero():
    """beta = 0 turns the target wrench off: every wrench t_j gives the same
    QP, min |G y|^2 over the friction pyramids with sum f_n >= gamma."""
    hand, obj, x, T, P = _sphere(8)
    ev = O.evaluate(O.Hand(hand), O.Object(obj), x, T, dict(P, beta=0.0))
    Q = ev["Q"]
    np.testing.assert_allclose(Q, Q[:, :1].repeat(Q.shape[1], 1), rtol=1e-9, atol=1e-14)
    # a zero force is infeasible (gamma > 0) but any feasible point bounds Q from above
    assert (Q >= -1e-15).all()
