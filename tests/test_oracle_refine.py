"""Pins for the oracle's refinement epilogue (fine / final stages,
Sec. IV-C Eqs. (10)-(11), SDF form)."""
import numpy as np
import pytest

import bodex_inputs as I
import oracle as O


def _case(kind):
    if kind == "sphere":
        hand, obj, x0, T, P, _, _ = I.workload("tiny", batch=6)
    else:
        hand = I.hand_template("hand5")
        obj = I.grid_object(2)
        x0 = I.initial_poses(hand, obj, 6, seed=12, gap=(-0.01, 0.005), flex=0.8)
        T, P = I.wrench_set(12), I.default_params()
    H, Ob = O.Hand(hand), O.Object(obj)
    pc = O.evaluate(H, Ob, x0, T, P)["p"] + 0.003  # coarse-stage points, offset so Q' is not zero
    return hand, obj, H, Ob, x0.astype(np.float64), pc


def _held_energy(hand, H, x, pc, kstar, targets, w_d, w_qp):
    """E with the sample choice and the targets p^f + delta n_out held fixed
    (Eq. (11)'s Detach), evaluated through the link frames."""
    frames = O.fk_frames(H, x)
    tips = hand.tip_samples.astype(np.float64)
    E = np.zeros(len(x))
    for b in range(len(x)):
        for i, link in enumerate(hand.contact_link):
            F = frames[b, link]
            c = F[:, :3] @ tips[i, kstar[b, i]] + F[:, 3]
            E[b] += w_d * ((c - targets[b, i]) ** 2).sum() + w_qp * ((c - pc[b, i]) ** 2).sum()
    return E


@pytest.mark.parametrize("kind", ["sphere", "grid"])
def test_refine_gradient_matches_differences(kind):
    hand, obj, H, Ob, x, pc = _case(kind)
    delta, w_d, w_qp = 0.01, 1000.0, 300.0
    r = O.refine_eval(H, Ob, x, pc, delta, w_d, w_qp)
    frames = O.fk_frames(H, x)
    tips = hand.tip_samples.astype(np.float64)
    targets = np.zeros((len(x), hand.n_contacts, 3))
    for b in range(len(x)):
        for i, link in enumerate(hand.contact_link):
            F = frames[b, link]
            cf = F[:, :3] @ tips[i, r["kstar"][b, i]] + F[:, 3]
            p, n, _, _ = O.contact(Ob, cf[None])
            targets[b, i] = p[0] - delta * n[0]
    np.testing.assert_allclose(_held_energy(hand, H, x, pc, r["kstar"], targets, w_d, w_qp), r["E"], rtol=1e-12)
    h = 1e-6
    g = np.zeros_like(x)
    for k in range(hand.dof):
        xp, xm = x.copy(), x.copy()
        xp[:, k] += h
        xm[:, k] -= h
        g[:, k] = (_held_energy(hand, H, xp, pc, r["kstar"], targets, w_d, w_qp)
                   - _held_energy(hand, H, xm, pc, r["kstar"], targets, w_d, w_qp)) / (2 * h)
    rel = np.linalg.norm(g - r["grad"], axis=1) / np.linalg.norm(g, axis=1)
    assert (rel < 1e-6).all(), rel


@pytest.mark.parametrize("kind", ["sphere", "grid"])
def test_refine_picks_the_lowest_sdf_sample(kind):
    hand, obj, H, Ob, x, pc = _case(kind)
    r = O.refine_eval(H, Ob, x, pc, 0.0, 1000.0, 0.0)
    frames = O.fk_frames(H, x)  # [B, n, 3, 4]
    tips = hand.tip_samples.astype(np.float64)
    Eref = np.zeros(len(x))
    for b in range(len(x)):
        for i, link in enumerate(hand.contact_link):
            F = frames[b, link]
            pts = tips[i] @ F[:, :3].T + F[:, 3]
            phi = O.sdf(Ob, pts)[0]
            k = int(np.argmin(phi))
            assert r["kstar"][b, i] == k
            # delta = 0, w_qp = 0: E is the paper's |c' - p^f|^2 summed
            p, n, ph, _ = O.contact(Ob, pts[k][None])
            Eref[b] += 1000.0 * float(((pts[k] - p[0]) ** 2).sum())
    np.testing.assert_allclose(r["E"], Eref, rtol=1e-12)


def test_refine_run_moves_toward_the_surface():
    hand, obj, H, Ob, x, pc = _case("sphere")
    P = I.default_params()
    E0 = O.refine_eval(H, Ob, x, pc, 0.01, P["w_d"], 0.0)["E"]
    x1, _, _, _ = O.refine_run(H, Ob, x, np.zeros_like(x), np.zeros_like(x), pc, 30, 0, 0.01, 0.0, P)
    E1 = O.refine_eval(H, Ob, x1, pc, 0.01, P["w_d"], 0.0)["E"]
    assert (E1 < E0).all()
