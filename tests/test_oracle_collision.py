"""Pins of the oracle's single-node collision: MRT + Guo forcing + recolouring (Sec. IV)."""
import numpy as np

import oracle as O


def feq(rho, u, c, w):
    cu = c @ u
    return w * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * u @ u)


def test_equilibrium_is_fixed_point():
    c, w, _ = O.lattice()
    rng = np.random.default_rng(1)
    for _ in range(5):
        rho, phi = rng.uniform(0.9, 1.1), rng.uniform(-1, 1)
        u = rng.uniform(-0.05, 0.05, 3)
        f = feq(rho, u, c, w)
        fa, fb = 0.5 * (1 + phi) * f, 0.5 * (1 - phi) * f
        om = rng.uniform(0.5, 1.9)
        fao, fbo, uo = O.collide_node(fa, fb, np.zeros(3), np.zeros(3), om, 8 * (2 - om) / (8 - om), 0.7)
        assert np.abs(fao - fa).max() < 1e-15
        assert np.abs(fbo - fb).max() < 1e-15
        assert np.abs(uo - u).max() < 1e-15


def test_conservation_and_force_increment():
    """Sum f* = Sum f, Sum c f* = Sum c f + F, and each component's mass is kept by
    the recolouring (sum_i w_i c_i/|c_i| = 0)."""
    c, w, _ = O.lattice()
    rng = np.random.default_rng(2)
    for _ in range(10):
        fa = rng.uniform(0.0, 0.1, 19)
        fb = rng.uniform(0.0, 0.1, 19)
        F = rng.uniform(-1e-3, 1e-3, 3)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        om = rng.uniform(0.5, 1.9)
        fao, fbo, _ = O.collide_node(fa, fb, F, n, om, 8 * (2 - om) / (8 - om), 0.7)
        assert abs(fao.sum() - fa.sum()) < 1e-15
        assert abs(fbo.sum() - fb.sum()) < 1e-15
        mom_in = c.T @ (fa + fb)
        mom_out = c.T @ (fao + fbo)
        assert np.abs(mom_out - (mom_in + F)).max() < 1e-15


def test_mrt_equals_two_relaxation_time_closed_form():
    """With the paper's S, M^-1 S M (f - feq) and M^-1 (I - S/2) M Fbar reduce to the
    TRT form f* = f - w(f+ - feq+) - w'(f- - feq-) + (1-w/2)Fbar+ + (1-w'/2)Fbar-.
    The TRT form is evaluated here from the lattice alone (no moment matrix)."""
    c, w, opp = O.lattice()
    rng = np.random.default_rng(3)
    for _ in range(10):
        fa = rng.uniform(0.0, 0.1, 19)
        fb = rng.uniform(0.0, 0.1, 19)
        F = rng.uniform(-1e-3, 1e-3, 3)
        om = rng.uniform(0.5, 1.9)
        omp = 8 * (2 - om) / (8 - om)
        f = fa + fb
        rho = f.sum()
        u = (c.T @ f + 0.5 * F) / rho
        fe = feq(rho, u, c, w)
        cu, cF = c @ u, c @ F
        Fb = w * (3 * cF + 9 * cu * cF - 3 * (u @ F))
        sym = lambda g: 0.5 * (g + g[opp])
        asym = lambda g: 0.5 * (g - g[opp])
        fs = f - om * sym(f - fe) - omp * asym(f - fe) + (1 - om / 2) * sym(Fb) + (1 - omp / 2) * asym(Fb)
        fao, fbo, _ = O.collide_node(fa, fb, F, np.zeros(3), om, omp, 0.7)
        # with n = 0 the recolouring only splits f* by the phase fractions
        assert np.abs((fao + fbo) - fs).max() < 1e-14
        assert np.abs(fao - fa.sum() / rho * fs).max() < 1e-14


def test_recolouring_perturbation():
    """f^a* - (rho^a/rho) f* = +beta rho^a rho^b/rho w_i (c_i.n)/|c_i| (Sec. IV recolouring)."""
    c, w, _ = O.lattice()
    rng = np.random.default_rng(4)
    fa = rng.uniform(0.0, 0.1, 19)
    fb = rng.uniform(0.0, 0.1, 19)
    n = np.array([0.3, -0.4, np.sqrt(1 - 0.25)])
    om = 1.2
    omp = 8 * (2 - om) / (8 - om)
    f0a, f0b, _ = O.collide_node(fa, fb, np.zeros(3), np.zeros(3), om, omp, 0.7)
    f1a, f1b, _ = O.collide_node(fa, fb, np.zeros(3), n, om, omp, 0.7)
    ra, rb = fa.sum(), fb.sum()
    norm = np.sqrt((c ** 2).sum(1))
    norm[0] = 1.0
    cos = (c @ n) / norm
    cos[0] = 0.0
    pert = 0.7 * ra * rb / (ra + rb) * w * cos
    assert np.abs((f1a - f0a) - pert).max() < 1e-15
    assert np.abs((f1b - f0b) + pert).max() < 1e-15
