"""Shared helpers for the GPU parity tests (inputs come from bodex_inputs,
expected values from the FP64 oracle; nothing here computes the method)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bodex_inputs as I  # noqa: E402
import oracle as O  # noqa: E402


def cuda(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    elif t.dtype == torch.float64:
        t = t.to(torch.float32)
    return t.cuda().contiguous()


def host(t):
    return t.detach().cpu().numpy()


def ineq_multiplier_l1(lam_ge):
    """1-norm of the oracle's multipliers (rows in a^T y >= b form)."""
    return np.abs(lam_ge).sum(-1)


def admm_rows(m, mu):
    """The ADMM constraint matrix A (9m+1 rows) and bounds, typed from the
    pyramid's definition for certificate arithmetic in the tests."""
    nv, nc = 3 * m, 9 * m + 1
    A = np.zeros((nc, nv))
    c8 = np.cos(np.pi / 8)
    for i in range(m):
        A[9 * i, 3 * i] = 1
        for k in range(8):
            ph = (2 * k + 1) * np.pi / 8
            A[9 * i + 1 + k, 3 * i:3 * i + 3] = (-mu * c8, np.cos(ph), np.sin(ph))
    A[9 * m, 0::3] = 1
    return A


def qp_certificate(G, T, y, z, lam, lam_star_l1, mu, beta, y_star):
    """Bounds on Q(y) - Q* from the ADMM point (y, z, lam) (all float64):
    with r_p = A y - z, r_d = P y + q + A^T lam and lam in the normal cone at z,
        -|lam*|_1 |r_p|_inf <= Q(y) - Q* <= |r_d|_inf |y* - y|_1 + |lam|_1 |r_p|_inf.
    Returns (lower, upper, rp, rd)."""
    m = G.shape[-1] // 3
    A = admm_rows(m, mu)
    P = 2 * np.einsum("bri,brj->bij", G, G)
    q = -2 * beta * np.einsum("bri,sr->bsi", G, T)
    rp = np.abs(np.einsum("ci,bsi->bsc", A, y) - z).max(-1)
    rd = np.abs(np.einsum("bij,bsj->bsi", P, y) + q + np.einsum("ci,bsc->bsi", A, lam)).max(-1)
    upper = rd * np.abs(y_star - y).sum(-1) + np.abs(lam).sum(-1) * rp
    lower = -lam_star_l1 * rp
    return lower, upper, rp, rd
