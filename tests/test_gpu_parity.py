"""GPU path vs the FP64 oracle, through the C ABI (one test per ABI call).

Tolerances (float32 path vs float64 oracle):
  * kinematics / SDF / G: absolute, from float32 rounding of chained
    transforms (positions ~0.1 m, so 2e-6 m is ~100 ulp);
  * voxel cell indices: bit-exact except near a face (|u - round(u)| < 1e-3);
  * QP value: |Q - Q*| <= 1e-4 |Q*| + 1e-6 for every QP (ADMM to 1e-6, then
    the exact FP64 polish); ADMM alone: inside the certificate interval
    computed from the GPU's own (y, z, lam) and the oracle's multipliers
    (see gpu_helpers), plus 1e-4 |Q*| + 1e-7;
  * forces: |dy|_inf <= 1e-3 where the oracle certifies the minimiser unique,
    and on the regularised QP (eps |y|^2, eps = 1e-3, same in both) for all;
  * energy and gradient: on the regularised QP, |dE| <= 1e-4 |E| + 1e-6 and
    |dgrad| / |grad| <= 1e-3 (the unregularised value function is not
    differentiable where the minimiser is not unique);
  * every QP of these tests converges to its residual target.
"""
import numpy as np
import pytest

from gpu_helpers import I, O, admm_rows, cuda, host, qp_certificate, torch

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


def qp_bar(Q_ref):
    """The QP-value tolerance: |dQ| <= 1e-4 |Q*| + 1e-6."""
    return 1e-4 * np.abs(Q_ref) + 1e-6


@pytest.mark.parametrize("wl,B", [("tiny", 64), ("paper_small", 96), ("paper_near", 64)])
def test_qp_value_within_1e4_relative(wl, B, request):
    """The unregularised QPs of Eqs. (7)-(9) at G from the oracle: ADMM to a
    1e-6 residual (K^-1 built in FP64), every QP converged, then polished
    (the exact minimum-norm-point solve in FP64): every QP's value within
    1e-4 |Q*| + 1e-6 of the oracle's exact active-set optimum, both as
    returned and recomputed from the returned forces."""
    hand, obj, x0, T, P = request.getfixturevalue(wl)
    G32 = _oracle_G(hand, obj, x0[:B], T, P)
    G = G32.astype(np.float64)
    ref = O.qp_solve(G, T, mu=MU, beta=BETA, gamma=GAMMA)
    assert (ref["status"] == 0).all() and ref["kkt"].max() < 1e-10
    prm = bx.qp_params(mu=MU, beta=BETA, gamma=GAMMA, eps_abs=1e-6, max_iter=100000, check_every=10, polish=1)
    out = bx.bodex_qp_solve_batch(cuda(G32), cuda(T), prm)
    st = host(out["status"])
    assert ((st & bx.ST_POLISHED) != 0).all() and ((st & bx.ST_NOT_CONVERGED) == 0).all()
    res = host(out["res"])  # the ADMM run's own residuals: every QP reached 1e-6
    assert (res <= 1e-6).all()
    y = host(out["y"]).astype(np.float64)
    Qy = ((BETA * T[None].astype(np.float64) - np.einsum("bri,bsi->bsr", G, y)) ** 2).sum(-1)
    bar = qp_bar(ref["Q"])
    assert (np.abs(host(out["Q"]) - ref["Q"]) <= bar).all()
    assert (np.abs(Qy - ref["Q"]) <= bar).all()
    # the returned forces are feasible: facets, 0 <= f_n <= 1, sum f_n >= gamma
    A = admm_rows(G.shape[-1] // 3, MU)
    Ay = np.einsum("ci,bsi->bsc", A, y)
    m = G.shape[-1] // 3
    assert (Ay[..., 9 * m] >= GAMMA - 1e-6).all()
    assert (Ay[..., 0:9 * m:9] >= -1e-6).all() and (Ay[..., 0:9 * m:9] <= 1 + 1e-6).all()
    facet = np.ones(9 * m, bool)
    facet[0::9] = False
    assert (Ay[..., :9 * m][..., facet] <= 1e-6).all()


@pytest.mark.parametrize("wl,B", [("tiny", 64), ("paper_small", 96), ("paper_near", 64)])
def test_qp_exact_solver_value_within_1e4_relative(wl, B, request):
    """qp.solver = EXACT (the float32 minimum-norm-point method, no ADMM):
    no QP stopped by the oracle-call cap; every QP's value within
    1e-4 |Q*| + 1e-6 of the oracle's; the Frank-Wolfe gap reported in
    res[..., 1] a valid upper bound on Q - Q* (to float32 rounding, 1e-6);
    forces feasible to 1e-6."""
    hand, obj, x0, T, P = request.getfixturevalue(wl)
    G32 = _oracle_G(hand, obj, x0[:B], T, P)
    G = G32.astype(np.float64)
    ref = O.qp_solve(G, T, mu=MU, beta=BETA, gamma=GAMMA)
    assert (ref["status"] == 0).all()
    prm = bx.qp_params(mu=MU, beta=BETA, gamma=GAMMA, max_iter=64, solver=bx.QP_EXACT)
    out = bx.bodex_qp_solve_batch(cuda(G32), cuda(T), prm)
    st = host(out["status"])
    assert (st == 0).all()
    y = host(out["y"]).astype(np.float64)
    Qy = ((BETA * T[None].astype(np.float64) - np.einsum("bri,bsi->bsr", G, y)) ** 2).sum(-1)
    bar = qp_bar(ref["Q"])
    assert (np.abs(host(out["Q"]) - ref["Q"]) <= bar).all()
    assert (np.abs(Qy - ref["Q"]) <= bar).all()
    gap = host(out["res"])[..., 1].astype(np.float64)
    assert (Qy - ref["Q"] <= gap + 1e-6).all()
    assert (host(out["iters"]) <= 64).all()
    m = G.shape[-1] // 3
    Ay = np.einsum("ci,bsi->bsc", admm_rows(m, MU), y)
    assert (Ay[..., 9 * m] >= GAMMA - 1e-6).all()
    assert (Ay[..., 0:9 * m:9] >= -1e-6).all() and (Ay[..., 0:9 * m:9] <= 1 + 1e-6).all()
    facet = np.ones(9 * m, bool)
    facet[0::9] = False
    assert (Ay[..., :9 * m][..., facet] <= 1e-6).all()
    # z is A y clamped to the bounds, lam is zero
    np.testing.assert_allclose(host(out["z"])[..., :9 * m][..., facet], np.minimum(Ay[..., :9 * m][..., facet], 0),
                               atol=1e-6)
    assert (host(out["lam"]) == 0).all()


@pytest.mark.parametrize("wl,B", [("tiny", 64), ("paper_small", 37), ("paper_near", 64)])
def test_qp_value_within_certificate(wl, B, request):
    """ADMM alone (no polishing) at a 1e-6 residual: every QP converges and
    its value lies inside the interval that the ADMM point (y, z, lam)
    certifies around Q* (gpu_helpers.qp_certificate), widened by
    1e-4 |Q*| + 1e-7 for float32 rounding."""
    hand, obj, x0, T, P = request.getfixturevalue(wl)
    G32 = _oracle_G(hand, obj, x0[:B], T, P)
    G = G32.astype(np.float64)
    ref = O.qp_solve(G, T, mu=MU, beta=BETA, gamma=GAMMA, want_lam=True)
    assert (ref["status"] == 0).all() and ref["kkt"].max() < 1e-10  # the oracle certified every QP
    prm = bx.qp_params(mu=MU, beta=BETA, gamma=GAMMA, eps_abs=1e-6, max_iter=100000, check_every=10)
    out = bx.bodex_qp_solve_batch(cuda(G32), cuda(T), prm)
    torch.cuda.synchronize()
    y, z, lam = (host(out[k]).astype(np.float64) for k in ("y", "z", "lam"))
    st = host(out["status"])
    assert ((st & bx.ST_NOT_CONVERGED) == 0).all()
    Qy = ((BETA * T[None].astype(np.float64) - np.einsum("bri,bsi->bsr", G, y)) ** 2).sum(-1)
    # the kernel's own Q is the float32 value of the same expression
    np.testing.assert_allclose(host(out["Q"]), Qy, rtol=1e-4, atol=1e-6)
    lo, hi, rp, rd = qp_certificate(G, T.astype(np.float64), y, z, lam, np.abs(ref["lam"]).sum(-1), MU, BETA,
                                    ref["y"])
    d = Qy - ref["Q"]
    tol = 1e-4 * np.abs(ref["Q"]) + 1e-7
    assert (d >= lo - tol).all(), (d - lo).min()
    assert (d <= hi + tol).all(), (d - hi).max()
    # residuals the kernel reports, and the same recomputed here in FP64 from
    # the returned float32 (y, z, lam)
    res = host(out["res"])
    assert (res[..., 0] <= 1e-6).all() and (res[..., 1] <= 1e-6).all()
    assert (rp <= 2e-6).all() and (rd <= 2e-6).all()


@pytest.mark.parametrize("wl,B", [("tiny", 64), ("paper_small", 96), ("paper_near", 64)])
def test_qp_forces_unique_unregularised(wl, B, request):
    """Forces of the unregularised QPs where the oracle certifies the
    minimiser unique (strict complementarity and a trivial null space of
    [G; A_active]): the polished forces (the exact FP64 solve) within 1e-3.
    ADMM's own forces are not compared here: "unique" admits minimisers whose
    defining matrix has singular values near 1e-5, where a 1e-6 residual
    leaves the ADMM forces far from y* (0.8 measured); forces of the ADMM
    path are compared on the regularised problem (below)."""
    hand, obj, x0, T, P = request.getfixturevalue(wl)
    G32 = _oracle_G(hand, obj, x0[:B], T, P)
    ref = O.qp_solve(G32.astype(np.float64), T, mu=MU, beta=BETA, gamma=GAMMA)
    uq = ref["unique"].astype(bool)
    assert uq.sum() >= 5
    prm = bx.qp_params(mu=MU, beta=BETA, gamma=GAMMA, eps_abs=1e-6, max_iter=100000, check_every=10, polish=1)
    y = host(bx.bodex_qp_solve_batch(cuda(G32), cuda(T), prm)["y"])
    assert np.abs(y - ref["y"])[uq].max() <= 1e-3


@pytest.mark.parametrize("m,s,B", [(3, 12, 21), (4, 6, 50), (5, 12, 33), (5, 1, 7), (4, 16, 9)])
def test_qp_forces_on_regularised_problem(m, s, B):
    """eps |y|^2 (eps = 1e-3, both sides) makes every minimiser unique: every
    QP converges to 1e-6 and its forces and residual wrench are within 1e-3."""
    T = I.wrench_set(12)[:s] if s <= 12 else np.concatenate([I.wrench_set(12), I.wrench_set(6)[:4]])
    p, n = I.random_contacts(B, m, seed=40 + m + s)
    G32 = O.grasp_matrix(p, n).astype(np.float32)
    G = G32.astype(np.float64)
    ref = O.qp_solve(G, T, eps_reg=1e-3)
    assert ref["unique"].all() and ref["kkt"].max() < 1e-10
    prm = bx.qp_params(eps_abs=1e-6, eps_reg=1e-3, max_iter=20000, check_every=10)
    out = bx.bodex_qp_solve_batch(cuda(G32), cuda(T), prm)
    y = host(out["y"])
    assert ((host(out["status"]) & bx.ST_NOT_CONVERGED) == 0).all()
    assert np.abs(y - ref["y"]).max() <= 1e-3
    r_gpu = T[None] - np.einsum("bri,bsi->bsr", G, y)
    r_ref = T[None] - np.einsum("bri,bsi->bsr", G, ref["y"])
    assert np.abs(r_gpu - r_ref).max() <= 1e-3


def test_qp_warm_start_and_edge_cases():
    T = I.wrench_set(6)
    p, n = I.random_contacts(13, 4, seed=5)  # 13: not a multiple of the grasps per CTA
    G32 = O.grasp_matrix(p, n).astype(np.float32)
    prm = bx.qp_params(eps_abs=1e-6, max_iter=100000, check_every=10)
    out = bx.bodex_qp_solve_batch(cuda(G32), cuda(T), prm)
    cold = host(out["iters"])
    prm.warm = 1
    again = bx.bodex_qp_solve_batch(cuda(G32), cuda(T), prm, y=out["y"].clone(), z=out["z"].clone(),
                                    lam=out["lam"].clone())
    # restarting at a converged point: y/z/lam reconstruct the iterate (up
    # to float32 rounding of z + lam / rho), so the restart needs a small
    # fraction of the cold iterations, and Q stays within 1e-6 (both points
    # lie within the 1e-6-residual certificate of Q*)
    it = host(again["iters"])
    assert ((host(again["status"]) & bx.ST_NOT_CONVERGED) == 0).all()
    assert np.median(it) <= 60 and it.max() <= cold.max() // 10
    np.testing.assert_allclose(host(again["Q"]), host(out["Q"]), atol=1e-6)
    # empty batch is a no-op; infeasible gamma is an error code
    e = bx.bodex_qp_solve_batch(cuda(G32[:0]), cuda(T), bx.qp_params())
    assert e["Q"].numel() == 0
    with pytest.raises(bx.BodexError) as ei:
        bx.bodex_qp_solve_batch(cuda(G32), cuda(T), bx.qp_params(gamma=5.0))
    assert ei.value.code == 4
    # fixed iteration count (eps_abs = 0) runs exactly max_iter iterations
    fixed = bx.bodex_qp_solve_batch(cuda(G32), cuda(T), bx.qp_params(max_iter=37))
    assert (host(fixed["iters"]) == 37).all()
    # the exact solver: empty batch, and the shapes it refuses
    e = bx.bodex_qp_solve_batch(cuda(G32[:0]), cuda(T), bx.qp_params(solver=bx.QP_EXACT))
    assert e["Q"].numel() == 0
    for bad in (dict(eps_reg=1e-3), dict(cone=bx.CONE_ELLIPTIC), dict(max_iter=0)):
        with pytest.raises(bx.BodexError) as ei:
            bx.bodex_qp_solve_batch(cuda(G32), cuda(T), bx.qp_params(solver=bx.QP_EXACT, **bad))
        assert ei.value.code == 1


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
    assert ((st & bx.ST_NOT_CONVERGED) == 0).all()  # every QP of every grasp reached 1e-6
    ok = np.ones(B, bool)
    if obj.kind != "sphere":  # queries within rounding of a voxel face may take the other cell
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


def test_three_fused_steps_match_oracle_adam(tiny):
    """Three upper iterations (Sec. IV-A; Adam and the clamp of Eq. (4)) in one
    fused launch against the oracle's run with its analytic gradient and
    exact QPs, on converged regularised QPs (eps_abs 1e-6, eps_reg 1e-3).
    Pose, first and second moments element by element; the Adam state's
    step counter is 3.  m and v are sums of the step gradients (weights 0.1
    ... and squares), so their error follows the gradient's (1e-3 relative
    at most, 1e-5 measured): per grasp |dm| <= 1e-4 |m| and |dv| <= 1e-4 |v|
    (2-norms), elementwise within 1e-4 relative plus 1e-5 of the grasp's
    largest entry.  The pose moves by lr m-hat / sqrt(v-hat) per step, a
    ratio of those sums, so |dx| <= 3 lr 1e-4 ~ 6e-6: asserted within 2e-6
    (rtol 1e-5 of x)."""
    hand, obj, x0, T, P = tiny
    Pr = dict(P, eps_reg=1e-3)
    H, Ob = bx.Hand(hand), bx.Object(obj)
    B = 32
    sp = bx.step_params(Pr, qp=bx.qp_params(eps_abs=1e-6, eps_reg=1e-3, max_iter=100000, check_every=10))
    st = bx.State(H, B, T.shape[0])
    st.set_pose(cuda(x0[:B]))
    stat = torch.zeros(B, dtype=torch.int32, device="cuda")
    bx.bodex_step(H, Ob, st, cuda(T), 3, sp, status=stat)
    assert ((host(stat) & (bx.ST_NOT_CONVERGED | bx.ST_NONFINITE)) == 0).all()
    xg = host(st.pose())
    mg, vg, t = st.adam()
    mg, vg = host(mg).astype(np.float64), host(vg).astype(np.float64)
    assert t == 3
    xo, mo, vo, _ = O.run(O.Hand(hand), O.Object(obj), x0[:B].astype(np.float64), T, Pr, n_steps=3,
                          grad_mode="analytic")
    np.testing.assert_allclose(xg, xo, rtol=1e-5, atol=2e-6)
    assert (np.linalg.norm(mg - mo, axis=1) <= 1e-4 * np.linalg.norm(mo, axis=1)).all()
    assert (np.linalg.norm(vg - vo, axis=1) <= 1e-4 * np.linalg.norm(vo, axis=1)).all()
    np.testing.assert_array_less(np.abs(mg - mo), 1e-4 * np.abs(mo) + 1e-5 * np.abs(mo).max(1, keepdims=True) + 1e-30)
    np.testing.assert_array_less(np.abs(vg - vo), 1e-4 * np.abs(vo) + 1e-5 * np.abs(vo).max(1, keepdims=True) + 1e-30)


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
