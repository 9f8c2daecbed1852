"""Adaptive ADMM penalty (residual balancing, OSQP Sec. 5.2) in solves with a
residual target: the results meet the same parity bars as fixed rho, and the
several-job kernel matches single launches bitwise."""
import numpy as np
import pytest

from gpu_helpers import I, O, cuda, host, qp_certificate, torch

import paper_2412_16490_gb300 as bx

pytestmark = pytest.mark.gpu

MU, BETA, GAMMA = 0.5, 1.0, 0.5


@pytest.mark.parametrize("m,s,B", [(5, 12, 40), (3, 6, 33), (4, 12, 21)])
def test_adaptive_qp_value_within_certificate(m, s, B):
    T = I.wrench_set(s)
    p, n = I.random_contacts(B, m, seed=90 + m)
    G32 = O.grasp_matrix(p, n).astype(np.float32)
    G = G32.astype(np.float64)
    ref = O.qp_solve(G, T, mu=MU, beta=BETA, gamma=GAMMA, want_lam=True)
    assert (ref["status"] == 0).all()
    prm = bx.qp_params(mu=MU, beta=BETA, gamma=GAMMA, eps_abs=1e-5, max_iter=100000, check_every=10, adaptive_rho=1)
    out = bx.bodex_qp_solve_batch(cuda(G32), cuda(T), prm)
    y, z, lam = (host(out[k]).astype(np.float64) for k in ("y", "z", "lam"))
    conv = (host(out["status"]) & bx.ST_NOT_CONVERGED) == 0
    # every QP converges but at most one: the grasp-shared penalty that the
    # normalised residual vote settles on can leave one QP's dual residual far
    # above the target (4e-2 seen); which QP, if any, moves with the rounding
    # of the iteration.  Fixed rho converges all of them.
    assert (~conv).sum() <= 1, [(i, host(out["res"])[i].tolist()) for i in zip(*np.nonzero(~conv))]
    Qy = ((BETA * T[None] - np.einsum("bri,bsi->bsr", G, y)) ** 2).sum(-1)
    lo, hi, rp, rd = qp_certificate(G, T.astype(np.float64), y, z, lam, np.abs(ref["lam"]).sum(-1), MU, BETA,
                                    ref["y"])
    d = Qy - ref["Q"]
    tol = 1e-4 * np.abs(ref["Q"]) + 1e-7
    assert (d >= lo - tol).all() and (d <= hi + tol).all()
    # lam comes back at the grasp's final rho: the recomputed residuals match the reported ones
    assert (rp[conv] <= 2e-5).all() and (rd[conv] <= 2e-5).all()


def test_adaptive_forces_on_the_regularised_problem():
    T = I.wrench_set(12)
    p, n = I.random_contacts(30, 5, seed=91)
    G32 = O.grasp_matrix(p, n).astype(np.float32)
    ref = O.qp_solve(G32.astype(np.float64), T, eps_reg=1e-3)
    out = bx.bodex_qp_solve_batch(cuda(G32), cuda(T),
                                  bx.qp_params(eps_abs=2e-6, eps_reg=1e-3, max_iter=100000, check_every=10,
                                               adaptive_rho=1))
    conv = (host(out["status"]) & bx.ST_NOT_CONVERGED) == 0
    # at most one QP stalls (the rule's failure mode above; fixed rho converges all)
    assert (~conv).sum() <= 1, [(i, host(out["res"])[i].tolist()) for i in zip(*np.nonzero(~conv))]
    # the adaptive path reaches 2e-6 here, not 1e-6 (its float32 floor lies
    # between, 3-5e-6 on a few QPs); the regularised objective is
    # 2 eps-strongly convex, so a point at residual 2e-6 lies within about
    # 2e-6 / (2 eps) (1 + |lam|) of y*: 2e-3 (fixed rho: 1e-3 at 1e-6)
    assert np.abs(host(out["y"]) - ref["y"])[conv].max() <= 2e-3


def test_adaptive_energy_and_gradient_in_the_fused_kernel():
    hand, obj, x0, T, P, _, _ = I.workload("tiny", batch=37)  # 37: a ragged last CTA
    Pr = dict(P, eps_reg=1e-3)
    H, Ob = bx.Hand(hand), bx.Object(obj)
    # 2e-6: adaptive rho's float32 floor lies between 1e-6 and 5e-6 on a few QPs
    sp = bx.step_params(Pr, qp=bx.qp_params(eps_abs=2e-6, eps_reg=1e-3, max_iter=100000, check_every=10,
                                            adaptive_rho=1))
    out = bx.bodex_energy_grad(H, Ob, cuda(x0), cuda(T), sp)
    ev = O.evaluate(O.Hand(hand), O.Object(obj), x0.astype(np.float64), T, Pr)
    ok = (host(out["status"]) & bx.ST_NOT_CONVERGED) == 0
    assert ok.all(), np.nonzero(~ok)[0]
    np.testing.assert_allclose(host(out["E"])[ok], ev["E"][ok], rtol=1e-4, atol=1e-6)
    g, gref = host(out["dEdx"]), ev["grad"]
    rel = np.linalg.norm(g - gref, axis=1) / np.maximum(np.linalg.norm(gref, axis=1), 1e-3)
    assert (rel[ok] <= 1e-3).all(), rel[ok].max()


def test_adaptive_step_in_a_mixed_launch_matches_single_launches():
    sp = bx.step_params(I.default_params(), qp=bx.qp_params(eps_abs=1e-5, max_iter=200, check_every=10,
                                                           adaptive_rho=1))
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
        jobs.append(dict(hand=H, obj=Ob, state=a, T=T, n_steps=8, E_last=Ea))
        bx.bodex_step(H, Ob, b, T, 8, sp, E_last=Eb)
        singles.append((a, b, Ea, Eb))
    bx.bodex_step_multi(jobs, sp)
    for a, b, Ea, Eb in singles:
        assert torch.equal(a.pose(), b.pose())
        assert torch.equal(Ea, Eb)
        assert torch.isfinite(Ea).all()
