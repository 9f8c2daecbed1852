"""GPU path vs the FP64 oracle, through the C ABI (one test per ABI call).

Tolerances (float32 path vs float64 oracle):
  * kinematics / SDF / G: absolute, from float32 rounding of chained
    transforms (positions ~0.1 m, so 2e-6 m is ~100 ulp);
  * voxel cell indices: bit-exact except near a face (|u - round(u)| < 1e-3);
  * QP value: inside the certificate interval computed from the GPU's own
    (y, z, lam) and the oracle's multipliers (see gpu_helpers), plus
    1e-4 |Q*| + 1e-7;
  * forces and gradients: on the regularised QP (eps |y|^2, eps = 1e-3,
    same in both), where the optimum is unique: |dy|_inf <= 1e-3 and
    |dgrad| / |grad| <= 1e-3.
"""
import numpy as np
import pytest

from gpu_helpers import I, O, cuda, host, qp_certificate, torch

import paper_2412_16490_gb300 as bx

pytestmark = pytest.mark.gpu

MU, BETA, GAMMA = 0.5, 1.0, 0.5


@pytest.fixture(scope="module")
def tiny():
    hand, obj, x0, T, P, _, _ = I.workload("tiny")
    return hand, obj, x0, T, P


@pytest.fixture(scope="module")
def paper_small():
    hand, obj, x0, T, P, _, _ = I.workload("paper", batch=96)
    return hand, obj, x0, T, P


@pytest.fixture(scope="module")
def paper_near():
    """Paper-scale hand and grid with poses taken from 40 oracle steps started
    near the surface, so that the queries fall inside the SDF grid."""
    hand, obj, _, T, P, _, _ = I.workload("paper", batch=1)
    x = I.initial_poses(hand, obj, 64, seed=11, gap=(-0.01, 0.005), flex=0.8)
    x, _, _, _ = O.run(O.Hand(hand), O.Object(obj), x, T, P, n_steps=40, grad_mode="analytic")
    return hand, obj, x.astype(np.float32), T, P


def off_voxel_faces(obj, c, tol=1e-3):
    """Per query: True unless an unclamped coordinate lies within `tol` voxels
    of a grid plane, or a coordinate sits within rounding of the box face
    (there the float32 and float64 paths may pick different cells)."""
    lo = obj.origin.astype(np.float64)
    hi = lo + obj.h * (obj.n - 1)
    inside = (c >= lo) & (c <= hi)
    u = (np.clip(c, lo, hi) - lo) / obj.h
    ok_in = np.abs(u - np.round(u)) > tol
    ok_out = np.minimum(np.abs(c - lo), np.abs(c - hi)) > tol * obj.h
    return np.where(inside, ok_in, ok_out).all(-1)


# ------------------------------------------------------------------ FK + contacts + G
@pytest.mark.parametrize("wl", ["tiny", "paper_small", "paper_near"])
def test_fk_contacts_matches_oracle(wl, request):
    hand, obj, x0, T, P = request.getfixturevalue(wl)
    H, Ob = bx.Hand(hand), bx.Object(obj)
    out = bx.bodex_fk_contacts(H, Ob, cuda(x0))
    torch.cuda.synchronize()
    ev = O.evaluate(O.Hand(hand), O.Object(obj), x0.astype(np.float64), T, P)
    c = host(out["c"])
    np.testing.assert_allclose(c, ev["c"], atol=2e-6)
    st = host(out["status"])
    assert (st & bx.ST_NONFINITE == 0).all()
    if obj.kind == "sphere":
        np.testing.assert_allclose(host(out["phi"]), ev["phi"], atol=2e-6)
        np.testing.assert_allclose(host(out["n"]), ev["n"], atol=2e-5)
        np.testing.assert_allclose(host(out["p"]), ev["p"], atol=2e-6)
        np.testing.assert_allclose(host(out["G"]), ev["G"], atol=5e-5)
        assert (host(out["cell"]) == 0).all()
        return
    far = off_voxel_faces(obj, ev["c"])
    assert far.mean() > 0.9
    cell = host(out["cell"])
    assert (cell[far] == ev["cell"][far]).all()  # bit-exact cell indices
    np.testing.assert_allclose(host(out["phi"])[far], ev["phi"][far], atol=5e-6)
    np.testing.assert_allclose(host(out["n"])[far], ev["n"][far], atol=2e-4)
    np.testing.assert_allclose(host(out["p"])[far], ev["p"][far], atol=5e-6)
    ok = far.all(-1)
    np.testing.assert_allclose(host(out["G"])[ok], ev["G"][ok], atol=2e-4)


def test_fk_contacts_edge_cases(tiny):
    hand, obj, x0, T, P = tiny
    H, Ob = bx.Hand(hand), bx.Object(obj)
    empty = bx.bodex_fk_contacts(H, Ob, cuda(x0[:0]))
    assert empty["c"].shape[0] == 0
    bad = x0[:3].copy()
    bad[1, 7] = np.nan
    st = host(bx.bodex_fk_contacts(H, Ob, cuda(bad))["status"])
    assert st[1] & bx.ST_NONFINITE and not (st[0] & bx.ST_NONFINITE)


# ------------------------------------------------------------------ batched QP
def _oracle_G(hand, obj, x0, T, P):
    ev = O.evaluate(O.Hand(hand), O.Object(obj), x0.astype(np.float64), T, P)
    return ev["G"].astype(np.float32)


@pytest.mark.parametrize("wl,B", [("tiny", 64), ("paper_small", 37), ("paper_near", 64)])
def test_qp_value_within_certificate(wl, B, request):
    hand, obj, x0, T, P = request.getfixturevalue(wl)
    G32 = _oracle_G(hand, obj, x0[:B], T, P)
    G = G32.astype(np.float64)
    ref = O.qp_solve(G, T, mu=MU, beta=BETA, gamma=GAMMA, want_lam=True)
    assert (ref["status"] == 0).all() and ref["kkt"].max() < 1e-10  # the oracle certified every QP
    prm = bx.qp_params(mu=MU, beta=BETA, gamma=GAMMA, eps_abs=1e-5, max_iter=20000, check_every=10)
    out = bx.bodex_qp_solve_batch(cuda(G32), cuda(T), prm)
    torch.cuda.synchronize()
    y, z, lam = (host(out[k]).astype(np.float64) for k in ("y", "z", "lam"))
    st = host(out["status"])
    conv = (st & bx.ST_NOT_CONVERGED) == 0
    assert conv.mean() > 0.97
    Qy = ((BETA * T[None].astype(np.float64) - np.einsum("bri,bsi->bsr", G, y)) ** 2).sum(-1)
    # the kernel's own Q is the float32 value of the same expression
    np.testing.assert_allclose(host(out["Q"]), Qy, rtol=1e-4, atol=1e-6)
    lo, hi, rp, rd = qp_certificate(G, T.astype(np.float64), y, z, lam, np.abs(ref["lam"]).sum(-1), MU, BETA,
                                    ref["y"])
    d = Qy - ref["Q"]
    tol = 1e-4 * np.abs(ref["Q"]) + 1e-7
    assert (d >= lo - tol).all(), (d - lo).min()
    assert (d <= hi + tol).all(), (d - hi).max()
    # on converged QPs the certificate is tight: Q within 3e-4 absolute
    assert np.abs(d[conv]).max() < 3e-4
    # residuals the kernel reports agree with the ones recomputed here
    res = host(out["res"])
    assert (res[..., 0][conv] <= 1e-5).all() and (res[..., 1][conv] <= 1e-5).all()
    assert (rp[conv] <= 2e-5).all() and (rd[conv] <= 2e-5).all()


@pytest.mark.parametrize("m,s,B", [(3, 12, 21), (4, 6, 50), (5, 12, 33), (5, 1, 7), (4, 16, 9)])
def test_qp_forces_on_regularised_problem(m, s, B):
    T = I.wrench_set(12)[:s] if s <= 12 else np.concatenate([I.wrench_set(12), I.wrench_set(6)[:4]])
    p, n = I.random_contacts(B, m, seed=40 + m + s)
    G32 = O.grasp_matrix(p, n).astype(np.float32)
    G = G32.astype(np.float64)
    ref = O.qp_solve(G, T, eps_reg=1e-3)
    assert ref["unique"].all() and ref["kkt"].max() < 1e-10
    prm = bx.qp_params(eps_abs=1e-6, eps_reg=1e-3, max_iter=20000, check_every=10)
    out = bx.bodex_qp_solve_batch(cuda(G32), cuda(T), prm)
    y = host(out["y"])
    conv = (host(out["status"]) & bx.ST_NOT_CONVERGED) == 0
    assert conv.mean() >= 0.95
    assert np.abs(y - ref["y"])[conv].max() <= 1e-3
    r_gpu = T[None] - np.einsum("bri,bsi->bsr", G, y)
    r_ref = T[None] - np.einsum("bri,bsi->bsr", G, ref["y"])
    assert np.abs(r_gpu - r_ref)[conv].max() <= 1e-3


def test_qp_warm_start_and_edge_cases():
    T = I.wrench_set(6)
    p, n = I.random_contacts(13, 4, seed=5)  # 13: not a multiple of the grasps per CTA
    G32 = O.grasp_matrix(p, n).astype(np.float32)
    prm = bx.qp_params(eps_abs=1e-5, max_iter=20000, check_every=10)
    out = bx.bodex_qp_solve_batch(cuda(G32), cuda(T), prm)
    cold = host(out["iters"])
    prm.warm = 1
    again = bx.bodex_qp_solve_batch(cuda(G32), cuda(T), prm, y=out["y"].clone(), z=out["z"].clone(),
                                    lam=out["lam"].clone())
    # restarting at a converged point: y/z/lam reconstruct the iterate, so
    # most QPs stop at the first check and none needs a cold-start budget
    it = host(again["iters"])
    assert np.median(it) <= 10 and (it <= np.maximum(cold, 10)).mean() > 0.9
    np.testing.assert_allclose(host(again["Q"]), host(out["Q"]), atol=1e-4)
    # empty batch is a no-op; infeasible gamma is an error code
    e = bx.bodex_qp_solve_batch(cuda(G32[:0]), cuda(T), bx.qp_params())
    assert e["Q"].numel() == 0
    with pytest.raises(bx.BodexError) as ei:
        bx.bodex_qp_solve_batch(cuda(G32), cuda(T), bx.qp_params(gamma=5.0))
    assert ei.value.code == 4
    # fixed iteration count (eps_abs = 0) runs exactly max_iter iterations
    fixed = bx.bodex_qp_solve_batch(cuda(G32), cuda(T), bx.qp_params(max_iter=37))
    assert (host(fixed["iters"]) == 37).all()


# ------------------------------------------------------------------ energy and gradient
@pytest.mark.parametrize("wl,B", [("tiny", 64), ("paper_small", 24), ("paper_near", 32)])
def test_energy_grad_matches_oracle(wl, B, request):
    hand, obj, x0, T, P = request.getfixturevalue(wl)
    x0 = x0[:B]
    Pr = dict(P, eps_reg=1e-3)
    H, Ob = bx.Hand(hand), bx.Object(obj)
    sp = bx.step_params(Pr, qp=bx.qp_params(eps_abs=1e-6, eps_reg=1e-3, max_iter=20000, check_every=10))
    out = bx.bodex_energy_grad(H, Ob, cuda(x0), cuda(T), sp)
    torch.cuda.synchronize()
    ev = O.evaluate(O.Hand(hand), O.Object(obj), x0.astype(np.float64), T, Pr)
    E, g = host(out["E"]), host(out["dEdx"])
    st = host(out["status"])
    assert (st & bx.ST_NONFINITE == 0).all()
    ok = (st & bx.ST_NOT_CONVERGED) == 0
    assert ok.mean() >= 0.9
    if obj.kind != "sphere":
        ok &= off_voxel_faces(obj, ev["c"]).all(-1)
        assert ok.sum() >= B // 2
    np.testing.assert_allclose(E[ok], ev["E"][ok], rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(host(out["Q"])[ok], ev["Q"][ok], atol=2e-5)
    gref = ev["grad"]
    rel = np.linalg.norm(g - gref, axis=1) / np.maximum(np.linalg.norm(gref, axis=1), 1e-3)
    assert (rel[ok] <= 1e-3).all(), rel[ok].max()


def test_step_is_adam_on_the_gradient(tiny):
    hand, obj, x0, T, P = tiny
    H, Ob = bx.Hand(hand), bx.Object(obj)
    B = 32
    sp = bx.step_params(P, qp=bx.qp_params(max_iter=30))
    x = cuda(x0[:B])
    g = host(bx.bodex_energy_grad(H, Ob, x, cuda(T), sp)["dEdx"])
    st = bx.State(H, B, T.shape[0])
    st.set_pose(x)
    E = torch.empty(B, device="cuda")
    bx.bodex_step(H, Ob, st, cuda(T), 1, sp, E_last=E)
    x1 = host(st.pose())
    lr = np.where(np.arange(hand.dof) < 3, P["lr_t"], P["lr_r"])
    want = np.clip(x0[:B] - lr * g / (np.abs(g) + P["adam_eps"]), hand.qmin, hand.qmax)
    np.testing.assert_allclose(x1, want, atol=2e-6)
    m, v, t = st.adam()
    assert t == 1
    np.testing.assert_allclose(host(m), 0.1 * g, rtol=1e-6, atol=1e-12)


def test_step_fused_launch_equals_repeated_launches(tiny):
    hand, obj, x0, T, P = tiny
    H, Ob = bx.Hand(hand), bx.Object(obj)
    B = 48
    sp = bx.step_params(P, qp=bx.qp_params(max_iter=30))
    a, b = bx.State(H, B, 6), bx.State(H, B, 6)
    a.set_pose(cuda(x0[:B]))
    b.set_pose(cuda(x0[:B]))
    bx.bodex_step(H, Ob, a, cuda(T), 5, sp)
    for _ in range(5):
        bx.bodex_step(H, Ob, b, cuda(T), 1, sp)
    assert torch.equal(a.pose(), b.pose())
    # and the run lowers the energy
    E0 = host(bx.bodex_energy_grad(H, Ob, cuda(x0[:B]), cuda(T), sp)["E"])
    E1 = host(bx.bodex_energy_grad(H, Ob, a.pose(), cuda(T), sp)["E"])
    assert np.median(E1 / E0) < 1.0
