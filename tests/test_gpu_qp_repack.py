"""The batched QP kernel repacks the QPs still running into the lowest warps
of the CTA at every residual check.  A QP's arithmetic must not depend on
which thread runs it: results are bitwise those of the same QP in another
batch (other CTA neighbours, so other repacking), with fixed and with
adaptive rho, and with a wrench count that leaves the last warp partial."""
import numpy as np
import pytest

from gpu_helpers import I, O, cuda, host, torch

import paper_2412_16490_gb300 as bx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,cone", [(5, 0), (3, 0), (4, 1), (5, 1)])
@pytest.mark.parametrize("s", [12, 7])
@pytest.mark.parametrize("adaptive", [0, 1])
def test_qp_results_do_not_depend_on_the_batch(m, cone, s, adaptive):
    """Also covers the wide form (the last QPs of a CTA, m lanes each): which
    QPs reach it, and when, depends on the batch."""
    T = cuda(I.wrench_set(12)[:s].copy())
    p, n = I.random_contacts(50, m, seed=95 + m)
    G = cuda(O.grasp_matrix(p, n).astype(np.float32))
    prm = bx.qp_params(eps_abs=1e-5, max_iter=3000, check_every=10, adaptive_rho=adaptive, cone=cone)
    full = bx.bodex_qp_solve_batch(G, T, prm)
    sub = bx.bodex_qp_solve_batch(G[3:41].contiguous(), T, prm)  # every grasp in another CTA position
    for k in ("y", "z", "lam", "Q", "iters", "status", "res"):
        assert torch.equal(full[k][3:41], sub[k]), k
    it = host(full["iters"])
    assert it.min() * 3 < it.max()  # iteration counts spread widely: QPs stop at different checks


def test_fixed_iteration_batch_runs_every_qp_to_the_cap():
    T = cuda(I.wrench_set(12))
    p, n = I.random_contacts(17, 4, seed=96)
    G = cuda(O.grasp_matrix(p, n).astype(np.float32))
    out = bx.bodex_qp_solve_batch(G, T, bx.qp_params(max_iter=37))
    assert (host(out["iters"]) == 37).all()
    assert (host(out["status"]) == 0).all()
    assert np.isfinite(host(out["Q"])).all() and (host(out["res"]) >= 0).all()


@pytest.mark.parametrize("B,s", [(1, 12), (1, 1), (200, 1), (13, 16), (0, 12)])
def test_qp_repacking_edge_shapes(B, s):
    """One grasp (a single partial warp: no wide form), one wrench per grasp
    (88 grasps per CTA, a partial last warp), the widest wrench set, and an
    empty batch: results match the same QPs solved one grasp at a time."""
    if s <= 12:
        T = I.wrench_set(12)[:s].copy()
    else:  # the 12 axes and unit force diagonals
        diag = np.zeros((s - 12, 6), np.float32)
        for k in range(s - 12):
            diag[k, k % 3], diag[k, (k + 1) % 3] = 0.6, 0.8
        T = np.concatenate([I.wrench_set(12), diag])
    T = cuda(T)
    p, n = I.random_contacts(max(B, 1), 5, seed=97)
    G = cuda(O.grasp_matrix(p, n).astype(np.float32))[:B].contiguous()
    prm = bx.qp_params(eps_abs=1e-5, max_iter=3000, check_every=10)
    full = bx.bodex_qp_solve_batch(G, T, prm)
    assert full["Q"].shape == (B, s)
    for b in range(0, B, max(1, B // 5)):
        one = bx.bodex_qp_solve_batch(G[b:b + 1].contiguous(), T, prm)
        for k in ("y", "z", "lam", "Q", "iters", "status"):
            assert torch.equal(full[k][b:b + 1], one[k]), (b, k)
