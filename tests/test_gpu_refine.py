"""Refinement epilogue (fine / final stages) on the GPU vs the FP64 oracle.
Sample choices k* are bit-exact except near ties (phi gap < 1e-6 m); one
step from the same state matches the oracle's Adam step."""
import numpy as np
import pytest

from gpu_helpers import I, O, cuda, host, torch

import paper_2412_16490_gb300 as bx

pytestmark = pytest.mark.gpu


def _case(kind, B):
    if kind == "sphere":
        hand, obj, x0, T, P, _, _ = I.workload("tiny", batch=B)
    else:
        hand = I.hand_template("hand5")
        obj = I.grid_object(2)
        x0 = I.initial_poses(hand, obj, B, seed=12, gap=(-0.01, 0.005), flex=0.8)
        T, P = I.wrench_set(12), I.default_params()
    H, Ob = O.Hand(hand), O.Object(obj)
    pc = (O.evaluate(H, Ob, x0, T, P)["p"] + 0.003).astype(np.float32)
    return hand, obj, x0, T, P, pc


@pytest.mark.parametrize("kind,B", [("sphere", 64), ("grid", 48)])
@pytest.mark.parametrize("delta", [0.01, 0.0])
def test_refine_step_matches_oracle(kind, B, delta):
    hand, obj, x0, T, P, pc = _case(kind, B)
    w_qp = 300.0
    H, Ob = bx.Hand(hand), bx.Object(obj)
    sp = bx.step_params(P)
    st = bx.State(H, B, T.shape[0])
    st.set_pose(cuda(x0))
    E = torch.empty(B, device="cuda")
    k = torch.empty((B, hand.n_contacts), dtype=torch.int32, device="cuda")
    bx.bodex_refine(H, Ob, st, cuda(pc), 1, delta, w_qp, sp, E_last=E, kstar=k)
    x1 = host(st.pose())
    ref = O.refine_eval(O.Hand(hand), O.Object(obj), x0.astype(np.float64), pc.astype(np.float64), delta,
                        P["w_d"], w_qp)
    tie = ref["gap"] < 1e-6
    kk = host(k)
    assert (kk[~tie] == ref["kstar"][~tie]).all()
    ok = ~tie.any(1)
    np.testing.assert_allclose(host(E)[ok], ref["E"][ok], rtol=2e-4, atol=1e-6)
    xr, _, _, _ = O.refine_run(O.Hand(hand), O.Object(obj), x0, np.zeros(x0.shape), np.zeros(x0.shape),
                               pc.astype(np.float64), 1, 0, delta, w_qp, P)
    # first Adam step is lr * sign(g); coordinates with a tiny gradient may differ in sign
    g = ref["grad"]
    big = (np.abs(g) > 1e-3 * np.abs(g).max(1, keepdims=True)) & ok[:, None]
    np.testing.assert_allclose(x1[big], xr[big], atol=2e-6)


def test_synthesize_three_stages():
    hand, obj, x0, T, P, _, _ = I.workload("tiny", batch=32)
    H, Ob = bx.Hand(hand), bx.Object(obj)
    sp = bx.step_params(P, qp=bx.qp_params(max_iter=30))
    out = bx.synthesize(H, Ob, cuda(x0), cuda(T), sp, coarse_steps=50, fine_steps=20, final_steps=20)
    xp, x, xs = host(out["x_p"]), host(out["x"]), host(out["x_s"])
    assert np.isfinite(x).all() and np.isfinite(xp).all()
    # x_s = 2 x - x_p (Sec. IV-D) from the library: 2 x is exact in float32, so bitwise
    np.testing.assert_array_equal(xs, (np.float32(2) * x - xp).astype(np.float32))
    # the final stage (no margin) ends closer to the surface than the pre-grasp
    ev_p = O.evaluate(O.Hand(hand), O.Object(obj), xp.astype(np.float64), T, P)
    ev_x = O.evaluate(O.Hand(hand), O.Object(obj), x.astype(np.float64), T, P)
    assert np.median(np.abs(ev_x["phi"] - hand.contact_radius)) < np.median(np.abs(ev_p["phi"] - hand.contact_radius)) + 1e-3
    # the metrics returned with the grasp are those of x
    ref = O.contact_metrics(O.Hand(hand), O.Object(obj), x.astype(np.float64))
    np.testing.assert_allclose(host(out["cdc"]), ref["cdc"], rtol=0, atol=4e-6)


def test_squeeze_pose_call_and_edge_cases():
    """bodex_squeeze_pose: bitwise 2 x - x_p on a ragged size, in place into x,
    an empty batch, and its error codes."""
    rng = np.random.default_rng(8)
    x = rng.normal(size=(1037, 28)).astype(np.float32)
    xp = rng.normal(size=(1037, 28)).astype(np.float32)
    got = host(bx.bodex_squeeze_pose(cuda(x), cuda(xp)))
    np.testing.assert_array_equal(got, (np.float32(2) * x - xp).astype(np.float32))
    xd = cuda(x)
    L = bx.load()
    import ctypes as C
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: C.c_void_p(t.data_ptr())
    assert L.bodex_squeeze_pose(ptr(xd), ptr(cuda(xp)), 1037, 28, ptr(xd), stream) == 0  # aliasing x
    np.testing.assert_array_equal(host(xd), got)
    assert bx.bodex_squeeze_pose(cuda(x[:0]), cuda(xp[:0])).shape == (0, 28)
    assert L.bodex_squeeze_pose(None, None, 3, 28, None, stream) == 1
    assert L.bodex_squeeze_pose(ptr(xd), ptr(xd), -1, 28, ptr(xd), stream) == 1


@pytest.mark.parametrize("kind,B", [("sphere", 64), ("grid", 200)])
@pytest.mark.parametrize("samples", [True, False])
def test_contact_metrics_match_oracle(kind, B, samples):
    """Signed fingertip distances and Contact Distance Consistency (Sec. V-B)
    vs the FP64 oracle.  The minimum over samples is continuous in the pose,
    so sample ties do not matter; FP32 chains at 0.1 m give 2e-6 m."""
    import dataclasses
    hand, obj, x0, _, _, _ = _case(kind, B)
    if not samples:
        hand = dataclasses.replace(hand, tip_samples=None)
    H, Ob = bx.Hand(hand), bx.Object(obj)
    out = bx.bodex_contact_metrics(H, Ob, cuda(x0))
    ref = O.contact_metrics(O.Hand(hand), O.Object(obj), x0.astype(np.float64))
    np.testing.assert_allclose(host(out["d"]), ref["d"], rtol=0, atol=2e-6)
    np.testing.assert_allclose(host(out["cdc"]), ref["cdc"], rtol=0, atol=4e-6)


def test_contact_metrics_ragged_batch_and_empty():
    hand, obj, x0, _, _, _ = _case("sphere", 37)  # ragged: 37 grasps over 16-grasp CTAs
    H, Ob = bx.Hand(hand), bx.Object(obj)
    out = bx.bodex_contact_metrics(H, Ob, cuda(x0))
    ref = O.contact_metrics(O.Hand(hand), O.Object(obj), x0.astype(np.float64))
    np.testing.assert_allclose(host(out["cdc"]), ref["cdc"], rtol=0, atol=4e-6)
    empty = bx.bodex_contact_metrics(H, Ob, cuda(x0[:0]))
    assert empty["d"].shape == (0, hand.n_contacts) and empty["cdc"].shape == (0,)
