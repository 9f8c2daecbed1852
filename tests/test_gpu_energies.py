"""Switchable comparison energies (Sec. V-C) on the GPU vs the FP64 oracle:
DFC (frictionless, equal unit normal forces: w_Q |G u|^2) and the QP
baseline (beta = 0).  Tolerances as in test_gpu_parity: E relative 1e-4,
gradient relative 1e-3 off voxel faces."""
import numpy as np
import pytest

from gpu_helpers import I, O, cuda, host, torch

import paper_2412_16490_gb300 as bx

pytestmark = pytest.mark.gpu


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


def _workload(kind, B):
    if kind == "tiny":
        hand, obj, x0, T, P, _, _ = I.workload("tiny", batch=B)
    else:
        hand, obj, _, T, P, _, _ = I.workload("paper", batch=1)
        x0 = I.initial_poses(hand, obj, B, seed=17, gap=(0.0, 0.01), flex=0.6)
    return hand, obj, x0, T, P


@pytest.mark.parametrize("kind,B", [("tiny", 64), ("paper", 48)])
def test_dfc_energy_and_gradient_match_oracle(kind, B):
    hand, obj, x0, T, P = _workload(kind, B)
    Pd = dict(P, energy=bx.ENERGY_DFC)
    H, Ob = bx.Hand(hand), bx.Object(obj)
    out = bx.bodex_energy_grad(H, Ob, cuda(x0), cuda(T), bx.step_params(Pd))
    ev = O.evaluate(O.Hand(hand), O.Object(obj), x0.astype(np.float64), T, dict(Pd, energy=O.ENERGY_DFC))
    ok = _off_faces(obj, ev["c"]).all(-1) if obj.kind != "sphere" else np.ones(B, bool)
    assert ok.sum() >= B // 2
    np.testing.assert_allclose(host(out["E"])[ok], ev["E"][ok], rtol=1e-4, atol=1e-6)
    assert (host(out["Q"]) == 0).all()
    g, gref = host(out["dEdx"]), ev["grad"]
    rel = np.linalg.norm(g - gref, axis=1) / np.maximum(np.linalg.norm(gref, axis=1), 1e-3)
    assert (rel[ok] <= 1e-3).all(), rel[ok].max()


def test_dfc_step_is_adam_on_the_dfc_gradient():
    hand, obj, x0, T, P = _workload("tiny", 32)
    Pd = dict(P, energy=bx.ENERGY_DFC)
    H, Ob = bx.Hand(hand), bx.Object(obj)
    sp = bx.step_params(Pd)
    x = cuda(x0)
    g = host(bx.bodex_energy_grad(H, Ob, x, cuda(T), sp)["dEdx"])
    st = bx.State(H, 32, T.shape[0])
    st.set_pose(x)
    E = torch.empty(32, device="cuda")
    bx.bodex_step(H, Ob, st, cuda(T), 1, sp, E_last=E)
    lr = np.where(np.arange(hand.dof) < 3, P["lr_t"], P["lr_r"])
    want = np.clip(x0 - lr * g / (np.abs(g) + P["adam_eps"]), hand.qmin, hand.qmax)
    np.testing.assert_allclose(host(st.pose()), want, atol=2e-6)
    ev = O.evaluate(O.Hand(hand), O.Object(obj), x0.astype(np.float64), T, dict(Pd, energy=O.ENERGY_DFC))
    np.testing.assert_allclose(host(E), ev["E"], rtol=1e-4, atol=1e-6)


def test_dfc_run_lowers_the_dfc_energy():
    hand, obj, x0, T, P = _workload("tiny", 64)
    Pd = dict(P, energy=bx.ENERGY_DFC)
    H, Ob = bx.Hand(hand), bx.Object(obj)
    sp = bx.step_params(Pd)
    E0 = host(bx.bodex_energy_grad(H, Ob, cuda(x0), cuda(T), sp)["E"])
    st = bx.State(H, 64, T.shape[0])
    st.set_pose(cuda(x0))
    E = torch.empty(64, device="cuda")
    bx.bodex_step(H, Ob, st, cuda(T), 100, sp, E_last=E)
    assert np.median(host(E) / E0) < 0.5


def test_qp_baseline_beta_zero_matches_oracle():
    hand, obj, x0, T, P = _workload("tiny", 48)
    Pr = dict(P, beta=0.0, eps_reg=1e-3)
    H, Ob = bx.Hand(hand), bx.Object(obj)
    sp = bx.step_params(Pr, qp=bx.qp_params(beta=0.0, eps_abs=1e-6, eps_reg=1e-3, max_iter=100000, check_every=10))
    out = bx.bodex_energy_grad(H, Ob, cuda(x0), cuda(T), sp)
    ev = O.evaluate(O.Hand(hand), O.Object(obj), x0.astype(np.float64), T, Pr)
    st = host(out["status"])
    ok = (st & bx.ST_NOT_CONVERGED) == 0
    assert ok.all(), np.nonzero(~ok)[0]
    np.testing.assert_allclose(host(out["E"])[ok], ev["E"][ok], rtol=1e-4, atol=1e-6)
    g, gref = host(out["dEdx"]), ev["grad"]
    rel = np.linalg.norm(g - gref, axis=1) / np.maximum(np.linalg.norm(gref, axis=1), 1e-3)
    assert (rel[ok] <= 1e-3).all(), rel[ok].max()
