"""The paper-scale workload at its full size (4096 grasps, 5-finger hand,
64^3 grid, 12 wrenches), in the launch configurations the bench times:
parity with the oracle on grasps sampled across the batch (the oracle
evaluates them one by one), and properties that hold at any size on every
grasp.  Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

from gpu_helpers import I, O, cuda, host, qp_certificate, torch

import paper_2412_16490_gb300 as bx

pytestmark = pytest.mark.gpu

MU, BETA, GAMMA = 0.5, 1.0, 0.5
SAMPLE = np.linspace(0, 4095, 48).round().astype(int)  # grasps spread over every CTA range


@pytest.fixture(scope="module")
def full():
    hand, obj, x0, T, P, steps, iters = I.workload("paper")
    assert x0.shape[0] == 4096 and T.shape[0] == 12 and (steps, iters) == (200, 50)
    return hand, obj, x0, T, P, bx.Hand(hand), bx.Object(obj)


def _off_faces(obj, c, tol=1e-3):
    lo = obj.origin.astype(np.float64)
    hi = lo + obj.h * (obj.n - 1)
    inside = (c >= lo) & (c <= hi)
    u = (np.clip(c, lo, hi) - lo) / obj.h
    return np.where(inside, np.abs(u - np.round(u)) > tol,
                    np.minimum(np.abs(c - lo), np.abs(c - hi)) > tol * obj.h).all(-1)


def test_fullsize_contacts_sampled(full):
    hand, obj, x0, T, P, H, Ob = full
    out = bx.bodex_fk_contacts(H, Ob, cuda(x0))
    assert (host(out["status"]) & bx.ST_NONFINITE == 0).all()  # every grasp
    ev = O.evaluate(O.Hand(hand), O.Object(obj), x0[SAMPLE].astype(np.float64), T, P)
    np.testing.assert_allclose(host(out["c"])[SAMPLE], ev["c"], atol=2e-6)
    far = _off_faces(obj, ev["c"])
    assert far.mean() > 0.9
    assert (host(out["cell"])[SAMPLE][far] == ev["cell"][far]).all()  # bit-exact cells
    np.testing.assert_allclose(host(out["phi"])[SAMPLE][far], ev["phi"][far], atol=5e-6)
    np.testing.assert_allclose(host(out["p"])[SAMPLE][far], ev["p"][far], atol=5e-6)
    ok = far.all(-1)
    np.testing.assert_allclose(host(out["G"])[SAMPLE][ok], ev["G"][ok], atol=2e-4)


def test_fullsize_qp_batch_sampled(full):
    """The bench's standalone QP configuration (all 49,152 QPs, cold start,
    1e-5, cap 5000, with the G the GPU computes), polished: every QP gets the
    exact FP64 solve, and the sampled grasps' values are within
    1e-4 |Q*| + 1e-6 of the oracle's.  The ADMM run's own residuals: the
    QPs it reports converged are at 1e-5, and on the sample their ADMM point
    (y before polishing, from the same launch without polish) lies inside
    its certificate around Q*."""
    hand, obj, x0, T, P, H, Ob = full
    G = bx.bodex_fk_contacts(H, Ob, cuda(x0))["G"]
    prm = bx.qp_params(mu=MU, beta=BETA, gamma=GAMMA, eps_abs=1e-5, max_iter=5000, check_every=10, polish=1)
    out = bx.bodex_qp_solve_batch(G, cuda(T), prm)
    st = host(out["status"])
    assert (st & bx.ST_NONFINITE == 0).all() and ((st & bx.ST_POLISHED) != 0).all()
    Gs = host(G)[SAMPLE].astype(np.float64)
    ref = O.qp_solve(Gs, T, mu=MU, beta=BETA, gamma=GAMMA, want_lam=True)
    assert (ref["status"] == 0).all()
    y = host(out["y"])[SAMPLE].astype(np.float64)
    Qy = ((BETA * T[None].astype(np.float64) - np.einsum("bri,bsi->bsr", Gs, y)) ** 2).sum(-1)
    bar = 1e-4 * np.abs(ref["Q"]) + 1e-6
    assert (np.abs(host(out["Q"])[SAMPLE] - ref["Q"]) <= bar).all()
    assert (np.abs(Qy - ref["Q"]) <= bar).all()
    # the same launch without polishing: ADMM's point and its certificate
    prm.polish = 0
    adm = bx.bodex_qp_solve_batch(G, cuda(T), prm)
    conv = (host(adm["status"]) & bx.ST_NOT_CONVERGED) == 0
    assert (host(adm["res"])[conv] <= 1e-5).all()
    assert torch.equal(adm["iters"], out["iters"]) and torch.equal(adm["res"], out["res"])
    ya, z, lam = (host(adm[k])[SAMPLE].astype(np.float64) for k in ("y", "z", "lam"))
    Qa = ((BETA * T[None].astype(np.float64) - np.einsum("bri,bsi->bsr", Gs, ya)) ** 2).sum(-1)
    lo, hi, rp, rd = qp_certificate(Gs, T.astype(np.float64), ya, z, lam, np.abs(ref["lam"]).sum(-1), MU, BETA,
                                    ref["y"])
    d = Qa - ref["Q"]
    tol = 1e-4 * np.abs(ref["Q"]) + 1e-7
    assert (d >= lo - tol).all() and (d <= hi + tol).all()


def test_fullsize_qp_batch_admm_then_exact_finish(full):
    """qp.polish = 2 on the bench's QP batch: ADMM to 1e-5 with a cap of 1000
    iterations, then the exact float32 solve of the QPs it left unconverged.
    Every QP ends converged or exactly solved; the converged ones are bit for
    bit those of the same ADMM run without the finish; the finished ones of
    the sampled grasps are within 1e-4 |Q*| + 1e-6 of the oracle's."""
    hand, obj, x0, T, P, H, Ob = full
    G = bx.bodex_fk_contacts(H, Ob, cuda(x0))["G"]
    prm = bx.qp_params(mu=MU, beta=BETA, gamma=GAMMA, eps_abs=1e-5, max_iter=1000, check_every=10, polish=2)
    out = bx.bodex_qp_solve_batch(G, cuda(T), prm)
    prm.polish = 0
    adm = bx.bodex_qp_solve_batch(G, cuda(T), prm)
    st, st0 = host(out["status"]), host(adm["status"])
    assert ((st & bx.ST_NOT_CONVERGED) == 0).all()
    fin = (st & bx.ST_POLISHED) != 0
    assert (fin == ((st0 & bx.ST_NOT_CONVERGED) != 0)).all()  # exactly the stragglers were finished
    assert 0 < fin.mean() < 0.5
    y, y0 = host(out["y"]), host(adm["y"])
    assert np.array_equal(y[~fin], y0[~fin]) and np.array_equal(host(out["Q"])[~fin], host(adm["Q"])[~fin])
    Gs = host(G)[SAMPLE].astype(np.float64)
    ref = O.qp_solve(Gs, T, mu=MU, beta=BETA, gamma=GAMMA)
    ys = y[SAMPLE].astype(np.float64)
    Qy = ((BETA * T[None].astype(np.float64) - np.einsum("bri,bsi->bsr", Gs, ys)) ** 2).sum(-1)
    bar = 1e-4 * np.abs(ref["Q"]) + 1e-6
    fs = fin[SAMPLE]
    assert fs.sum() >= 10
    assert (np.abs(Qy - ref["Q"])[fs] <= bar[fs]).all()


def test_fullsize_qp_batch_exact_solver(full):
    """The same 49,152 QPs with qp.solver = EXACT: no QP stopped by the cap,
    and the sampled grasps' values within 1e-4 |Q*| + 1e-6 of the oracle's."""
    hand, obj, x0, T, P, H, Ob = full
    G = bx.bodex_fk_contacts(H, Ob, cuda(x0))["G"]
    out = bx.bodex_qp_solve_batch(G, cuda(T), bx.qp_params(mu=MU, beta=BETA, gamma=GAMMA, max_iter=64,
                                                            solver=bx.QP_EXACT))
    st = host(out["status"])
    assert (st == 0).all()
    Gs = host(G)[SAMPLE].astype(np.float64)
    ref = O.qp_solve(Gs, T, mu=MU, beta=BETA, gamma=GAMMA)
    y = host(out["y"])[SAMPLE].astype(np.float64)
    Qy = ((BETA * T[None].astype(np.float64) - np.einsum("bri,bsi->bsr", Gs, y)) ** 2).sum(-1)
    bar = 1e-4 * np.abs(ref["Q"]) + 1e-6
    assert (np.abs(Qy - ref["Q"]) <= bar).all()
    assert (np.abs(host(out["Q"])[SAMPLE] - ref["Q"]) <= bar).all()


def test_fullsize_energy_gradient_sampled(full):
    hand, obj, x0, T, P, H, Ob = full
    Pr = dict(P, eps_reg=1e-3)
    sp = bx.step_params(Pr, qp=bx.qp_params(eps_abs=1e-6, eps_reg=1e-3, max_iter=100000, check_every=10))
    out = bx.bodex_energy_grad(H, Ob, cuda(x0), cuda(T), sp)
    st = host(out["status"])
    assert (st & bx.ST_NONFINITE == 0).all() and np.isfinite(host(out["dEdx"])).all()
    assert ((st & bx.ST_NOT_CONVERGED) == 0).all()  # every QP of all 4096 grasps reached 1e-6
    ev = O.evaluate(O.Hand(hand), O.Object(obj), x0[SAMPLE].astype(np.float64), T, Pr)
    ok = _off_faces(obj, ev["c"]).all(-1)  # queries within rounding of a voxel face may take the other cell
    assert ok.sum() >= len(SAMPLE) // 2
    np.testing.assert_allclose(host(out["E"])[SAMPLE][ok], ev["E"][ok], rtol=1e-4, atol=1e-6)
    g, gref = host(out["dEdx"])[SAMPLE], ev["grad"]
    rel = np.linalg.norm(g - gref, axis=1) / np.maximum(np.linalg.norm(gref, axis=1), 1e-3)
    assert (rel[ok] <= 1e-3).all(), rel[ok].max()


def test_fullsize_step_launch(full):
    """The bench's fused step (50 ADMM iterations) on every grasp: the first
    step is Adam on the evaluated gradient; a 5-step launch equals five
    1-step launches bitwise; the 200-step run lowers the energy."""
    hand, obj, x0, T, P, H, Ob = full
    sp = bx.step_params(P, qp=bx.qp_params(max_iter=50))
    x, Td = cuda(x0), cuda(T)
    g = host(bx.bodex_energy_grad(H, Ob, x, Td, sp)["dEdx"])
    st = bx.State(H, 4096, 12)
    st.set_pose(x)
    bx.bodex_step(H, Ob, st, Td, 1, sp)
    lr = np.where(np.arange(hand.dof) < 3, P["lr_t"], P["lr_r"])
    want = np.clip(x0 - lr * g / (np.abs(g) + P["adam_eps"]), hand.qmin, hand.qmax)
    np.testing.assert_allclose(host(st.pose()), want, atol=2e-6)
    a, b = bx.State(H, 4096, 12), bx.State(H, 4096, 12)
    a.set_pose(x)
    b.set_pose(x)
    bx.bodex_step(H, Ob, a, Td, 5, sp)
    for _ in range(5):
        bx.bodex_step(H, Ob, b, Td, 1, sp)
    assert torch.equal(a.pose(), b.pose())
    E = torch.empty(4096, device="cuda")
    status = torch.empty(4096, dtype=torch.int32, device="cuda")
    c = bx.State(H, 4096, 12)
    c.set_pose(x)
    bx.bodex_step(H, Ob, c, Td, 200, sp, E_last=E, status=status)
    assert (host(status) & bx.ST_NONFINITE == 0).all()
    E0 = host(bx.bodex_energy_grad(H, Ob, x, Td, sp)["E"])
    assert np.median(host(E) / E0) < 0.5


def test_fullsize_mixed_launch_equals_single_launches():
    """The mixed-template batch at full size (8704 grasps over 6 jobs, 3-, 4-
    and 5-contact hands): one several-job launch of 5 upper steps gives every
    grasp the pose of its own job's launch, bitwise."""
    jobs, T = I.mixed_workload(seed=4)
    assert sum(x.shape[0] for _, _, x in jobs) == 8704
    Td = cuda(T)
    sp = bx.step_params(I.default_params(), qp=bx.qp_params(max_iter=50))
    hands, table, singles = {}, [], []
    for hand, obj, x0 in jobs:
        H = hands.setdefault(hand.name, bx.Hand(hand))
        Ob = bx.Object(obj)
        a, b = bx.State(H, x0.shape[0], 12), bx.State(H, x0.shape[0], 12)
        a.set_pose(cuda(x0))
        b.set_pose(cuda(x0))
        table.append(dict(hand=H, obj=Ob, state=a, T=Td, n_steps=5))
        bx.bodex_step(H, Ob, b, Td, 5, sp)
        singles.append((a, b))
    bx.bodex_step_multi(table, sp)
    for a, b in singles:
        assert torch.equal(a.pose(), b.pose())
