"""The fused step and evaluation with the exact lower level
(qp.solver = EXACT: every QP of every upper step solved by the float32
minimum-norm-point method, warm-started from the previous step's working
set), through the C ABI, against the FP64 oracle and against itself.

Tolerances: energy |dE| <= 1e-4 |E| + 1e-6 and every wrench's Q within
1e-4 |Q*| + 1e-6 (the QP-value bar), on grasps whose queries keep off voxel
faces.  The unregularised gradient is not compared with the oracle: where a
minimiser is not unique the value function is not differentiable (Danskin).
"""
import numpy as np
import pytest

from gpu_helpers import I, O, cuda, host, torch

import paper_2412_16490_gb300 as bx

pytestmark = pytest.mark.gpu


def _exact(P, iters=64):
    return bx.step_params(P, qp=bx.qp_params(max_iter=iters, solver=bx.QP_EXACT))


def _off_faces(obj, c, tol=1e-3):
    if obj.kind == "sphere":
        return np.ones(c.shape[:-1], bool).all(-1)
    lo = obj.origin.astype(np.float64)
    hi = lo + obj.h * (obj.n - 1)
    inside = (c >= lo) & (c <= hi)
    u = (np.clip(c, lo, hi) - lo) / obj.h
    return np.where(inside, np.abs(u - np.round(u)) > tol,
                    np.minimum(np.abs(c - lo), np.abs(c - hi)) > tol * obj.h).all(-1).all(-1)


@pytest.mark.parametrize("wl,B", [("tiny", 64), ("paper", 48)])
def test_exact_evaluation_matches_oracle(wl, B):
    hand, obj, x0, T, P, _, _ = I.workload(wl, batch=B)
    H, Ob = bx.Hand(hand), bx.Object(obj)
    out = bx.bodex_energy_grad(H, Ob, cuda(x0), cuda(T), _exact(P))
    ev = O.evaluate(O.Hand(hand), O.Object(obj), x0.astype(np.float64), T, P)
    st = host(out["status"])
    assert ((st & (bx.ST_NONFINITE | bx.ST_NOT_CONVERGED)) == 0).all()
    ok = _off_faces(obj, ev["c"])
    assert ok.sum() >= B // 2
    Q = host(out["Q"])
    assert (np.abs(Q - ev["Q"])[ok] <= 1e-4 * np.abs(ev["Q"][ok]) + 1e-6).all()
    E = host(out["E"])
    np.testing.assert_allclose(E[ok], ev["E"][ok], rtol=1e-4, atol=1e-6)
    assert np.isfinite(host(out["dEdx"])).all()


def test_exact_step_launch_equals_repeated_launches_and_lowers_energy():
    """The working sets carry over between steps through the state: one
    launch of 6 steps equals six 1-step launches bitwise, and the run lowers
    the energy."""
    hand, obj, x0, T, P, _, _ = I.workload("tiny", batch=48)
    H, Ob = bx.Hand(hand), bx.Object(obj)
    sp = _exact(P)
    a, b = bx.State(H, 48, T.shape[0]), bx.State(H, 48, T.shape[0])
    a.set_pose(cuda(x0))
    b.set_pose(cuda(x0))
    bx.bodex_step(H, Ob, a, cuda(T), 6, sp)
    for _ in range(6):
        bx.bodex_step(H, Ob, b, cuda(T), 1, sp)
    assert torch.equal(a.pose(), b.pose())
    assert torch.equal(a.adam()[0], b.adam()[0])
    E0 = host(bx.bodex_energy_grad(H, Ob, cuda(x0), cuda(T), sp)["E"])
    st = bx.State(H, 48, T.shape[0])
    st.set_pose(cuda(x0))
    E = torch.empty(48, device="cuda")
    stat = torch.zeros(48, dtype=torch.int32, device="cuda")
    bx.bodex_step(H, Ob, st, cuda(T), 50, sp, E_last=E, status=stat)
    assert ((host(stat) & (bx.ST_NONFINITE | bx.ST_NOT_CONVERGED)) == 0).all()
    assert np.median(host(E) / E0) < 0.5
    # the residual the state reports is each grasp's largest Frank-Wolfe gap at the last step
    assert (host(st.residual()) <= 1e-4).all()


def test_exact_warm_start_gives_the_same_energy_as_a_cold_solve():
    """After a few steps, the warm-started solves' energies equal a cold
    exact evaluation at the same poses (to the QP-value bar)."""
    hand, obj, x0, T, P, _, _ = I.workload("tiny", batch=32)
    H, Ob = bx.Hand(hand), bx.Object(obj)
    sp = _exact(P)
    st = bx.State(H, 32, T.shape[0])
    st.set_pose(cuda(x0))
    bx.bodex_step(H, Ob, st, cuda(T), 5, sp)
    x5 = st.pose()
    # step 6's energy is evaluated at x5 with the warm corrals
    E = torch.empty(32, device="cuda")
    bx.bodex_step(H, Ob, st, cuda(T), 1, sp, E_last=E)
    cold = bx.bodex_energy_grad(H, Ob, x5, cuda(T), sp)
    np.testing.assert_allclose(host(E), host(cold["E"]), rtol=1e-4, atol=1e-6)


def test_exact_several_job_launch_equals_single_launches():
    jobs, T = I.mixed_workload(seed=4, scale=1 / 32)
    P = I.default_params()
    sp = _exact(P)
    Tt = cuda(T)
    hands, single, multi = {}, [], []
    for hand, obj, x0 in jobs:
        Hj = hands.setdefault(hand.name, bx.Hand(hand))
        Ob = bx.Object(obj)
        for lst in (single, multi):
            st = bx.State(Hj, x0.shape[0], T.shape[0])
            st.set_pose(cuda(x0))
            lst.append(dict(hand=Hj, obj=Ob, state=st, T=Tt, n_steps=7))
    for j in single:
        bx.bodex_step(j["hand"], j["obj"], j["state"], Tt, 7, sp)
    bx.bodex_step_multi(multi, sp)
    for a, b in zip(single, multi):
        assert torch.equal(a["state"].pose(), b["state"].pose())


@pytest.mark.parametrize("m,s,B", [(3, 12, 21), (4, 6, 50), (5, 1, 7), (4, 16, 9), (5, 12, 1)])
def test_exact_qp_shapes_match_oracle(m, s, B):
    """The standalone exact solver over hand sizes, wrench counts from 1 to
    16 and ragged batches (B not a multiple of a block's grasps)."""
    T = I.wrench_set(12)[:s] if s <= 12 else np.concatenate([I.wrench_set(12), I.wrench_set(6)[:4]])
    p, n = I.random_contacts(B, m, seed=60 + m + s)
    G32 = O.grasp_matrix(p, n).astype(np.float32)
    ref = O.qp_solve(G32.astype(np.float64), T)
    out = bx.bodex_qp_solve_batch(cuda(G32), cuda(T), bx.qp_params(max_iter=64, solver=bx.QP_EXACT))
    assert (host(out["status"]) == 0).all()
    assert (np.abs(host(out["Q"]) - ref["Q"]) <= 1e-4 * np.abs(ref["Q"]) + 1e-6).all()


def test_admm_then_exact_finish_small_batch():
    """qp.polish = 2 on a ragged batch: every QP converged by ADMM or exactly
    finished, the finished ones within the QP-value bar; without a status
    array the call is refused."""
    T = I.wrench_set(12)
    p, n = I.random_contacts(37, 5, seed=77)
    G32 = O.grasp_matrix(p, n).astype(np.float32)
    ref = O.qp_solve(G32.astype(np.float64), T)
    prm = bx.qp_params(eps_abs=1e-5, max_iter=150, check_every=10, polish=2)
    out = bx.bodex_qp_solve_batch(cuda(G32), cuda(T), prm)
    st = host(out["status"])
    assert ((st & bx.ST_NOT_CONVERGED) == 0).all()
    fin = (st & bx.ST_POLISHED) != 0
    assert fin.any()
    assert (np.abs(host(out["Q"]) - ref["Q"])[fin] <= (1e-4 * np.abs(ref["Q"]) + 1e-6)[fin]).all()
    import ctypes as C
    L = bx.load()
    Gd, Td = cuda(G32), cuda(T)
    y, z, lam, Q = (torch.zeros(sh, device="cuda") for sh in ((37, 12, 15), (37, 12, 46), (37, 12, 46), (37, 12)))
    ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
    rc = L.bodex_qp_solve_batch(ptr(Gd), 37, 5, ptr(Td), 12, C.byref(prm), ptr(y), ptr(z), ptr(lam), ptr(Q), None, None,
                                None, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1
