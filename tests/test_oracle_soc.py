"""Pins for the elliptic-cone oracle (the unlinearised friction model the
pyramid of Sec. IV-A approximates): Q* is bracketed by exact QPs over the
K-facet pyramids inscribed in (Q_in >= Q*) and circumscribed about
(Q_out <= Q*) the cone."""
import numpy as np
import pytest

import bodex_inputs as I
import oracle as O

K = 256


def _antipodal(r=0.04):
    """Two contacts at +-r x with inward normals -+x."""
    p = np.array([[[r, 0.0, 0.0], [-r, 0.0, 0.0]]])
    n = np.array([[[-1.0, 0.0, 0.0], [1.0, 0.0, 0.0]]])
    return p, n


@pytest.mark.parametrize("beta", [0.3, 0.8, 1.0, 1.6])
def test_antipodal_tangential_demand_closed_form(beta):
    """A tangential demand beta along y: each contact carries at most mu f_n
    <= mu of friction in any tangential direction (the cone is round), the
    normals must cancel and the torques too, so Q* = max(0, beta - 2 mu)^2."""
    mu = 0.5
    p, n = _antipodal()
    G = O.grasp_matrix(p, n)
    T = np.array([[0.0, 1.0, 0.0, 0.0, 0.0, 0.0]])
    r = O.qp_soc(G, T, mu=mu, beta=beta, gamma=0.5, K=K)
    want = max(0.0, beta - 2 * mu) ** 2
    assert (r["status"] == 0).all()
    assert r["Q_out"][0, 0] <= want + 1e-12
    assert r["Q_in"][0, 0] >= want - 1e-12
    assert r["Q_in"][0, 0] - r["Q_out"][0, 0] <= 4 * (1 - np.cos(np.pi / K)) + 1e-12


def test_bracket_survives_a_turn_of_the_tangent_basis():
    """The cone is round, so turning every contact's (d, e) basis by any angle
    leaves Q* unchanged while the polyhedral brackets move: all of them must
    contain one common value."""
    p, n = I.random_contacts(12, 4, seed=9)
    G = O.grasp_matrix(p, n)
    T = I.wrench_set(6)
    lo, hi = None, None
    for th in (0.0, 0.3, 0.77, 1.9):
        Gr = G.copy()
        c, s = np.cos(th), np.sin(th)
        for i in range(4):
            d, e = G[:, :, 3 * i + 1].copy(), G[:, :, 3 * i + 2].copy()
            Gr[:, :, 3 * i + 1] = c * d + s * e
            Gr[:, :, 3 * i + 2] = -s * d + c * e
        r = O.qp_soc(Gr, T, K=K)
        assert (r["status"] == 0).all()
        lo = r["Q_out"] if lo is None else np.maximum(lo, r["Q_out"])
        hi = r["Q_in"] if hi is None else np.minimum(hi, r["Q_in"])
    assert (lo <= hi + 1e-12).all(), (lo - hi).max()


def test_cone_lies_between_the_eight_facet_pyramids():
    """Q_soc <= Q over the inscribed 8-facet pyramid of Sec. IV-A, whose edges
    are vertices of the inscribed K-gon; and the optimum of the cone is a
    feasible point of the circumscribed 8-facet pyramid."""
    p, n = I.random_contacts(10, 5, seed=4)
    G = O.grasp_matrix(p, n)
    T = I.wrench_set(12)
    r = O.qp_soc(G, T, K=K)
    pyr = O.qp_solve(G, T)
    assert (r["Q_in"] <= pyr["Q"] + 1e-9).all()
    circ = O.qp_solve(G, T, mu=0.5 / np.cos(np.pi / 8))
    assert (circ["Q"] <= r["Q_out"] + 1e-9).all()


def test_inscribed_point_is_cone_feasible_and_multipliers_are_stationary():
    p, n = I.random_contacts(6, 5, seed=2)
    G = O.grasp_matrix(p, n)
    T = I.wrench_set(12)
    mu, beta, gamma = 0.5, 1.0, 0.5
    r = O.qp_soc(G, T, mu=mu, beta=beta, gamma=gamma, K=K)
    y = r["y"]
    fn, fd, fe = y[..., 0::3], y[..., 1::3], y[..., 2::3]
    assert (np.hypot(fd, fe) <= mu * fn + 1e-12).all()
    assert (fn >= -1e-12).all() and (fn <= 1 + 1e-12).all() and (fn.sum(-1) >= gamma - 1e-12).all()
    # grad f + A_row^T lam = 0 (row form: f_n, cone rows (mu f_n, f_d, f_e), sum row)
    lam = r["lam"]
    for b in range(G.shape[0]):
        for j in range(T.shape[0]):
            g = 2 * G[b].T @ (G[b] @ y[b, j] - beta * T[j])
            l = lam[b, j]
            at = np.zeros(15)
            for i in range(5):
                at[3 * i] = l[4 * i] + mu * l[4 * i + 1] + l[20]
                at[3 * i + 1] = l[4 * i + 2]
                at[3 * i + 2] = l[4 * i + 3]
            assert np.abs(g + at).max() < 1e-9
