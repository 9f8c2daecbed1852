"""Pins for the oracle's lower-level QP (Sec. IV-A, Eqs. (7)-(9)).

The oracle's active-set solver is checked against things it does not share
code paths with: hand-derived closed forms on antipodal contacts, brute-force
enumeration of the faces of the feasible set (m <= 3), KKT certificates,
and invariances the problem must have.
"""
import json
import math
import os

import numpy as np
import pytest

import bodex_inputs as I
import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def _G_explicit(p, n, d, e):
    """Grasp matrix of Eq. (2) typed from its definition, for explicit bases."""
    cols = []
    for pi, ni, di, ei in zip(p, n, d, e):
        for v in (ni, di, ei):
            cols.append(np.concatenate([v, np.cross(pi, v)]))
    return np.array(cols).T  # 6 x 3m


def _antipodal(r, rot):
    pA, nA = np.array([r, 0, 0.0]), np.array([-1.0, 0, 0])
    pB, nB = -pA, -nA
    dA, eA = np.array([0, 1.0, 0]), np.array([0, 0, -1.0])
    dB, eB = np.array([0, 1.0, 0]), np.array([0, 0, 1.0])
    c, s = math.cos(rot), math.sin(rot)
    dA, eA = c * dA + s * eA, -s * dA + c * eA
    dB, eB = c * dB + s * eB, -s * dB + c * eB
    assert np.allclose(np.cross(dA, eA), nA) and np.allclose(np.cross(dB, eB), nB)
    return _G_explicit([pA, pB], [nA, nB], [dA, dB], [eA, eB])


def test_antipodal_closed_forms():
    fx = json.load(open(os.path.join(HERE, "golden", "antipodal_closed_forms.json")))
    for case in fx["cases"]:
        G = _antipodal(fx["r"], case["rot"])[None]
        T = np.array(case["wrench"], float)[None]
        out = O.qp_solve(G, T, mu=fx["mu"], beta=case["beta"], gamma=case["gamma"])
        assert out["status"][0, 0] == 0
        assert out["kkt"][0, 0] < 1e-10, case["name"]
        assert abs(out["Q"][0, 0] - case["Q"]) < 1e-12, (case["name"], out["Q"][0, 0], case["Q"])
        Qb, _ = O.qp_bruteforce(G, T, mu=fx["mu"], beta=case["beta"], gamma=case["gamma"])
        assert abs(Qb[0, 0] - case["Q"]) < 1e-12, (case["name"], Qb[0, 0])


@pytest.mark.parametrize("m,seed", [(1, 11), (2, 12), (3, 13)])
@pytest.mark.parametrize("beta,gamma", [(1.0, 0.5), (0.5, 0.1), (2.0, 1.0), (1.2, 0.5)])
def test_active_set_matches_bruteforce(m, seed, beta, gamma):
    B = {1: 16, 2: 12, 3: 3}[m]
    T = I.wrench_set(6)
    p, n = I.random_contacts(B, m, seed)
    G = O.grasp_matrix(p, n)
    out = O.qp_solve(G, T, beta=beta, gamma=gamma)
    if gamma > m:
        assert (out["status"] == 2).all()
        return
    Qb, yb = O.qp_bruteforce(G, T, beta=beta, gamma=gamma)
    assert np.isfinite(Qb).all()
    np.testing.assert_allclose(out["Q"], Qb, rtol=0, atol=1e-11)
    assert out["kkt"].max() < 1e-10
    # where the optimum is certified unique the two routes agree on y too
    u = out["unique"].astype(bool)
    if u.any():
        np.testing.assert_allclose(out["y"][u], yb[u], atol=1e-8)


@pytest.mark.parametrize("m,s", [(4, 6), (5, 12)])
def test_kkt_certificates(m, s):
    T = I.wrench_set(s)
    p, n = I.random_contacts(48, m, 100 + m)
    G = O.grasp_matrix(p, n)
    out = O.qp_solve(G, T)
    assert (out["status"] == 0).all()
    assert out["kkt"].max() < 1e-10
    y = out["y"]
    # feasibility of every returned force, checked on the cone of Eq. (1)
    # linearised: 0 <= f_n <= 1, |f_t| <= mu f_n (inscribed pyramid is inside)
    fn, fd, fe = y[..., 0::3], y[..., 1::3], y[..., 2::3]
    assert (fn >= -1e-12).all() and (fn <= 1 + 1e-12).all()
    assert (np.hypot(fd, fe) <= 0.5 * fn + 1e-12).all()
    assert (fn.sum(-1) >= 0.5 - 1e-12).all()
    # Q is the residual of the returned forces
    W = 1.0 * T[None] - np.einsum("brk,bsk->bsr", G, y)
    np.testing.assert_allclose(out["Q"], (W ** 2).sum(-1), atol=1e-12)


def test_invariances():
    m, B = 4, 24
    T = I.wrench_set(12)
    p, n = I.random_contacts(B, m, 7)
    G = O.grasp_matrix(p, n)
    base = O.qp_solve(G, T)["Q"]
    # 8-fold symmetry: turning one contact's basis by pi/4 about n
    G2 = G.copy()
    c, s = math.cos(math.pi / 4), math.sin(math.pi / 4)
    d, e = G[:, :, 3 * 1 + 1].copy(), G[:, :, 3 * 1 + 2].copy()
    G2[:, :, 4], G2[:, :, 5] = c * d + s * e, -s * d + c * e
    np.testing.assert_allclose(O.qp_solve(G2, T)["Q"], base, atol=1e-11)
    # permutation of contacts
    perm = [2, 0, 3, 1]
    cols = np.concatenate([[3 * k, 3 * k + 1, 3 * k + 2] for k in perm])
    np.testing.assert_allclose(O.qp_solve(G[:, :, cols], T)["Q"], base, atol=1e-11)
    # a smaller gamma enlarges the feasible set: Q cannot increase
    Qg = O.qp_solve(G, T, gamma=0.1)["Q"]
    assert (Qg <= base + 1e-12).all()
    # bound from the feasible point y = (gamma/m) normal pushes
    y0 = np.zeros(3 * m)
    y0[0::3] = 0.5 / m
    ub = ((T[None] - np.einsum("brk,k->br", G, y0)[:, None, :]) ** 2).sum(-1)
    assert (base <= ub + 1e-12).all()
    # beta = 0 (QP_baseline energy, Sec. V-C) gives Q >= 0 and no larger than
    # the residual of the same feasible point
    Q0 = O.qp_solve(G, T, beta=0.0)["Q"]
    ub0 = (np.einsum("brk,k->br", G, y0) ** 2).sum(-1)
    assert (Q0 >= -1e-15).all() and (Q0 <= ub0[:, None] + 1e-12).all()


def test_eps_reg_makes_unique():
    T = I.wrench_set(6)
    p, n = I.random_contacts(16, 4, 21)
    G = O.grasp_matrix(p, n)
    out = O.qp_solve(G, T, eps_reg=1e-6)
    assert out["kkt"].max() < 1e-10
    assert out["unique"].mean() > 0.9
    plain = O.qp_solve(G, T)["Q"]
    # the regulariser moves Q by at most eps * |y|^2 <= eps * 2m
    assert (out["Q"] - plain >= -1e-12).all() and (out["Q"] - plain <= 1e-6 * 8 + 1e-12).all()


def test_infeasible_gamma():
    T = I.wrench_set(6)
    p, n = I.random_contacts(2, 2, 3)
    G = O.grasp_matrix(p, n)
    out = O.qp_solve(G, T, gamma=2.5)
    assert (out["status"] == 2).all()


def test_active_set_certifies_a_stress_batch():
    """Every solve ends at a KKT point (residual <= 1e-10) across contact
    counts, wrench sets, (beta, gamma) and normal noise levels."""
    for m in (3, 4, 5):
        for s in (6, 12):
            T = I.wrench_set(s)
            for seed, (beta, gamma) in enumerate(((1.0, 0.5), (0.5, 1.0), (2.0, 0.1))):
                p, n = I.random_contacts(48, m, seed=500 + 10 * m + seed, spread=0.6 if seed % 2 else 1.0,
                                         normal_noise=0.05 + 0.1 * seed)
                out = O.qp_solve(O.grasp_matrix(p, n), T, beta=beta, gamma=gamma)
                assert (out["status"] == 0).all()
                assert out["kkt"].max() < 1e-10
