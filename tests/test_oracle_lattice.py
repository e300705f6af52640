"""Pins of the oracle's lattice, moment basis and relaxation rates (Sec. IV)."""
import itertools
import json
import math
import os

import numpy as np

import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_d3q19_weights_and_isotropy():
    c, w, opp = O.lattice()
    assert c.shape == (19, 3)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs((w[:, None] * c).sum(0)).max() == 0.0
    second = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.abs(second - np.eye(3) / 3.0).max() < 1e-15
    # fourth-order isotropy: sum w c_a c_b c_c c_d = (d_ab d_cd + d_ac d_bd + d_ad d_bc)/9
    d = np.eye(3)
    for a, b, cc, dd in itertools.product(range(3), repeat=4):
        s = (w * c[:, a] * c[:, b] * c[:, cc] * c[:, dd]).sum()
        ref = (d[a, b] * d[cc, dd] + d[a, cc] * d[b, dd] + d[a, dd] * d[b, cc]) / 9.0
        assert abs(s - ref) < 1e-15
    for i in range(19):
        assert (c[opp[i]] == -c[i]).all()
    # all 19 velocities distinct, |c|^2 in {0,1,2}
    assert len({tuple(v) for v in c}) == 19
    assert set((c ** 2).sum(1)) == {0, 1, 2}


def test_mrt_basis_orthogonal_and_conserved_rows():
    c, w, _ = O.lattice()
    M, Mi, S = O.mrt_matrices()
    G = M @ M.T
    assert np.abs(G - np.diag(np.diag(G))).max() < 1e-12
    assert np.abs(M @ Mi - np.eye(19)).max() < 1e-12
    assert (M[0] == 1).all()
    for row, ax in ((3, 0), (5, 1), (7, 2)):
        assert (M[row] == c[:, ax]).all()
    # the conserved moments (density, momentum) are exactly those with S = 0
    assert set(np.where(S == 0)[0]) == {0, 3, 5, 7}


def test_relaxation_pattern_is_two_relaxation_time():
    """Every non-conserved moment even in c relaxes with omega, every odd one with
    omega': the paper's S is a two-relaxation-time operator."""
    c, _, opp = O.lattice()
    M, _, S = O.mrt_matrices()
    for k in range(19):
        even = np.allclose(M[k][opp], M[k])
        odd = np.allclose(M[k][opp], -M[k])
        assert even or odd
        if S[k] == 1:
            assert even
        elif S[k] == 2:
            assert odd


def test_magic_parameter_three_sixteenths():
    for omega in np.linspace(0.2, 1.95, 15):
        op = 8.0 * (2.0 - omega) / (8.0 - omega)
        lam = (1.0 / omega - 0.5) * (1.0 / op - 0.5)
        assert abs(lam - GOLD["omega_prime_magic"]["value"]) < 1e-14


def test_recolouring_constant_k_matches_paper():
    """k = (1/2) sum_i w_i c_ix^2/|c_i| = (1+sqrt2)/18 ~ 0.134 (Sec. V F)."""
    c, w, _ = O.lattice()
    norm = np.sqrt((c ** 2).sum(1))
    k = 0.5 * sum(w[i] * c[i, 0] ** 2 / norm[i] for i in range(1, 19))
    assert abs(k - (1 + math.sqrt(2)) / 18) < 1e-15
    assert abs(k - GOLD["k_d3q19"]["value"]) < GOLD["k_d3q19"]["tol"]


def test_harmonic_viscosity():
    kw = dict(nu_a=1.0 / 6.0, nu_b=1.0 / 60.0, rho0=1.0)
    for phi, nu in ((1.0, 1.0 / 6.0), (-1.0, 1.0 / 60.0)):
        om = O.omega_of_phi(phi, 1.0, **kw)
        assert abs((1.0 / om - 0.5) / 3.0 - nu) < 1e-15
    # phi = 0: harmonic mean of the two viscosities
    om = O.omega_of_phi(0.0, 1.0, **kw)
    eta = (1.0 / om - 0.5) / 3.0
    assert abs(eta - 2.0 / (6.0 + 60.0)) < 1e-15
    # tau uses the local density: eta = rho cs2 (tau - 1/2)
    om = O.omega_of_phi(1.0, 1.2, **kw)
    assert abs(1.2 / 3.0 * (1.0 / om - 0.5) - 1.0 / 6.0) < 1e-15
