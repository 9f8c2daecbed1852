"""Mixed-template persistent launch (bodex_step_multi): jobs with hand
templates of m = 3, 4, 5 contacts, different objects, batch sizes and step
counts in one launch give each job the result it gets alone."""
import numpy as np
import pytest

from gpu_helpers import I, cuda, host, torch

import paper_2412_16490_gb300 as bx

pytestmark = pytest.mark.gpu


def _jobs():
    specs = [("hand3", I.grid_object(4, n=48), 37, 5), ("hand4x4", I.sphere_object(), 50, 7),
             ("hand5", I.grid_object(2), 29, 3), ("hand4", I.grid_object(6, n=56), 11, 6)]
    out = []
    for k, (name, obj, B, n) in enumerate(specs):
        hand = I.hand_template(name)
        x0 = I.initial_poses(hand, obj, B, seed=30 + k)
        out.append(dict(tpl=hand, objd=obj, x0=x0, B=B, n=n))
    return out


def test_multi_launch_matches_single_launches():
    T = cuda(I.wrench_set(12))
    sp = bx.step_params(I.default_params(), qp=bx.qp_params(max_iter=30))
    jobs = _jobs()
    for j in jobs:
        j["hand"], j["obj"] = bx.Hand(j["tpl"]), bx.Object(j["objd"])
        j["mix"], j["alone"] = bx.State(j["hand"], j["B"], 12), bx.State(j["hand"], j["B"], 12)
        j["mix"].set_pose(cuda(j["x0"]))
        j["alone"].set_pose(cuda(j["x0"]))
    bx.bodex_step_multi([dict(hand=j["hand"], obj=j["obj"], state=j["mix"], T=T, n_steps=j["n"]) for j in jobs], sp)
    for j in jobs:
        bx.bodex_step(j["hand"], j["obj"], j["alone"], T, j["n"], sp)
    torch.cuda.synchronize()
    for j in jobs:
        a, b = host(j["mix"].pose()), host(j["alone"].pose())
        np.testing.assert_array_equal(a, b, err_msg=j["tpl"].name)
        assert j["mix"].adam()[2] == j["n"]


def test_cta_tile_does_not_change_results():
    hand, obj, x0, T, P, _, _ = I.workload("paper", batch=70)
    H, Ob = bx.Hand(hand), bx.Object(obj)
    poses = []
    for g in (2, 4, 8, 0):
        sp = bx.step_params(P, qp=bx.qp_params(max_iter=20), grasps_per_cta=g)
        st = bx.State(H, 70, 12)
        st.set_pose(cuda(x0))
        bx.bodex_step(H, Ob, st, cuda(T), 4, sp)
        poses.append(st.pose())
    for p in poses[1:]:
        assert torch.equal(p, poses[0])


def test_residual_output_tracks_admm_iterations():
    hand, obj, x0, T, P, _, _ = I.workload("tiny", batch=40)
    H, Ob = bx.Hand(hand), bx.Object(obj)
    res = []
    for iters in (5, 200):
        st = bx.State(H, 40, 6)
        st.set_pose(cuda(x0))
        bx.bodex_step(H, Ob, st, cuda(T), 3, bx.step_params(P, qp=bx.qp_params(max_iter=iters)))
        res.append(host(st.residual()))
    assert np.isfinite(res[0]).all() and (res[0] > 0).all()
    assert np.median(res[1]) < 0.2 * np.median(res[0])


def test_multi_launch_rejects_bad_tables():
    hand = I.hand_template("hand4")
    H, Ob = bx.Hand(hand), bx.Object(I.sphere_object())
    st = bx.State(H, 4, 6)
    T = cuda(I.wrench_set(12))  # s = 12 does not match the state's s = 6
    with pytest.raises(bx.BodexError):
        bx.bodex_step_multi([dict(hand=H, obj=Ob, state=st, T=T, n_steps=1)], bx.step_params())
    bx.bodex_step_multi([], bx.step_params())  # empty table is a no-op


@pytest.mark.parametrize("solver", ["admm", "exact"])
def test_work_pulling_launch_equals_single_launches(solver):
    """step_params.work_pulling = 1: a persistent grid pulling the jobs' tiles
    (costliest first) from an atomic counter gives every job the result of
    its own launch: bitwise with ADMM; with the exact solve within float32
    rounding (the item loop changes the compiler's multiply-add contraction
    in the kinematics and adjoint code; 5e-8 measured after 3 steps).  The
    default one-CTA-per-tile launch is bitwise in both."""
    T = cuda(I.wrench_set(12))
    qp = bx.qp_params(max_iter=30) if solver == "admm" else bx.qp_params(max_iter=64, solver=bx.QP_EXACT)
    jobs = _jobs()
    for j in jobs:
        j["hand"], j["obj"] = bx.Hand(j["tpl"]), bx.Object(j["objd"])
        for k in ("pull", "once", "alone"):
            j[k] = bx.State(j["hand"], j["B"], 12)
            j[k].set_pose(cuda(j["x0"]))
    for k, wp in (("pull", 1), ("once", 0)):
        sp = bx.step_params(I.default_params(), qp=qp, work_pulling=wp)
        bx.bodex_step_multi([dict(hand=j["hand"], obj=j["obj"], state=j[k], T=T, n_steps=j["n"]) for j in jobs], sp)
    for j in jobs:
        bx.bodex_step(j["hand"], j["obj"], j["alone"], T, j["n"], bx.step_params(I.default_params(), qp=qp))
    for j in jobs:
        if solver == "admm":
            assert torch.equal(j["pull"].pose(), j["alone"].pose()), j["tpl"].name
        else:
            np.testing.assert_allclose(host(j["pull"].pose()), host(j["alone"].pose()), rtol=0, atol=1e-5)
        assert torch.equal(j["once"].pose(), j["alone"].pose()), j["tpl"].name


@pytest.mark.parametrize("wp", [0, 1])
def test_several_job_launch_with_empty_and_idle_jobs(wp):
    """Jobs with no grasps or no steps are skipped in both schedules; the
    others get their own launch's result; a launch of no jobs is a no-op."""
    T = cuda(I.wrench_set(12))
    sp = bx.step_params(I.default_params(), qp=bx.qp_params(max_iter=20), work_pulling=wp)
    hand = I.hand_template("hand5")
    H, Ob = bx.Hand(hand), bx.Object(I.grid_object(2))
    x0 = I.initial_poses(hand, I.grid_object(2), 19, seed=3)
    empty, idle, real, alone = bx.State(H, 0, 12), bx.State(H, 19, 12), bx.State(H, 19, 12), bx.State(H, 19, 12)
    for st in (idle, real, alone):
        st.set_pose(cuda(x0))
    bx.bodex_step_multi([dict(hand=H, obj=Ob, state=empty, T=T, n_steps=5),
                         dict(hand=H, obj=Ob, state=idle, T=T, n_steps=0),
                         dict(hand=H, obj=Ob, state=real, T=T, n_steps=5)], sp)
    bx.bodex_step(H, Ob, alone, T, 5, sp)
    assert torch.equal(real.pose(), alone.pose())
    assert torch.equal(idle.pose(), cuda(x0)) and idle.adam()[2] == 0
    bx.bodex_step_multi([], sp)
