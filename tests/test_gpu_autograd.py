"""torch.autograd binding (forward: fused QP solve, backward: the
hand-written adjoint kernel) against the FP64 oracle's central differences
(h = 1e-6) on 64 sampled instances of the 1024-grasp gradient workload."""
import numpy as np
import pytest

from gpu_helpers import I, O, cuda, host, torch

import paper_2412_16490_gb300 as bx
from paper_2412_16490_gb300.autograd import grasp_energy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def grad_case():
    hand, obj, x0, T, P, _, _ = I.workload("grad")
    P = dict(P, eps_reg=1e-3)
    # 2e-6: one QP of the 6144 (grasp 505, wrench 0) has its float32 dual-residual
    # floor at 1.9e-6 and never reaches 1e-6; at 2e-6 every QP converges
    sp = bx.step_params(P, qp=bx.qp_params(eps_abs=2e-6, eps_reg=1e-3, max_iter=100000, check_every=10))
    return hand, obj, x0, T, P, sp, bx.Hand(hand), bx.Object(obj)


def test_autograd_gradient_matches_oracle_differences(grad_case):
    hand, obj, x0, T, P, sp, H, Ob = grad_case
    x = cuda(x0).requires_grad_(True)
    E = grasp_energy(x, H, Ob, cuda(T), sp)
    assert E.shape == (1024,)
    E.sum().backward()
    g = host(x.grad)
    idx = np.random.default_rng(3).choice(1024, 64, replace=False)
    gfd = O.grad_fd(O.Hand(hand), O.Object(obj), x0[idx].astype(np.float64), T, P, step=1e-6)
    rel = np.linalg.norm(g[idx] - gfd, axis=1) / np.maximum(np.linalg.norm(gfd, axis=1), 1e-3)
    # the envelope gradient holds at the optimum: every QP of every grasp
    # reached the residual target (the forward's status bits)
    st = host(bx.bodex_energy_grad(H, Ob, cuda(x0), cuda(T), sp)["status"])
    assert ((st & bx.ST_NOT_CONVERGED) == 0).all(), np.nonzero(st & bx.ST_NOT_CONVERGED)[0]
    assert (rel <= 1e-3).all(), np.sort(rel)[-5:]
    assert np.median(rel) <= 1e-4


def test_adjoint_kernel_equals_fused_gradient(grad_case):
    hand, obj, x0, T, P, sp, H, Ob = grad_case
    x, Tt = cuda(x0[:200]), cuda(T)
    fwd = bx.bodex_energy_grad(H, Ob, x, Tt, sp)
    adj = bx.bodex_energy_adjoint(H, Ob, x, Tt, sp, fwd["y"])
    np.testing.assert_allclose(host(adj["E"]), host(fwd["E"]), rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(host(adj["dEdx"]), host(fwd["dEdx"]), rtol=1e-5, atol=1e-6)


def test_backward_applies_the_incoming_weights(grad_case):
    hand, obj, x0, T, P, sp, H, Ob = grad_case
    x = cuda(x0[:64]).requires_grad_(True)
    w = torch.linspace(-2.0, 3.0, 64, device="cuda")
    (w * grasp_energy(x, H, Ob, cuda(T), sp)).sum().backward()
    fwd = bx.bodex_energy_grad(H, Ob, cuda(x0[:64]), cuda(T), sp)
    np.testing.assert_allclose(host(x.grad), host(w[:, None] * fwd["dEdx"]), rtol=1e-5, atol=1e-5)
