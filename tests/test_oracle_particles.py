"""Pins of the oracle's fluid-particle coupling (Sec. V A-C, E)."""
import math

import numpy as np

import oracle as O


def test_solid_marking_brute_force():
    """A node is inside particle p iff |x - x_p|^2 < R_p^2 (minimum image)."""
    nx, ny, nz = 20, 18, 16
    s = O.OracleSim(nx, ny, nz, wall_z0=1)
    xp, R = (18.3, 2.7, 7.1), 4.6  # straddles the periodic x and y boundaries
    s.add_particle(xp, R, kinematic=True)
    own = s.owner().reshape(nz, ny, nx)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if z == 0:
                    assert own[z, y, x] == 1
                    continue
                d = [(x - xp[0] + nx / 2) % nx - nx / 2, (y - xp[1] + ny / 2) % ny - ny / 2, z - xp[2]]
                inside = d[0] ** 2 + d[1] ** 2 + d[2] ** 2 < R * R
                assert own[z, y, x] == (2 if inside else 0)


def test_sphere_in_fluid_at_rest_feels_no_force():
    n = 20
    s = O.OracleSim(n, n, n)
    s.init_fields(np.ones(n ** 3))
    s.add_particle((10.0, 10.0, 10.0), 5.0, kinematic=True)
    s.step(3)
    P = s.particles()[0]
    assert np.abs(P[0:6]).max() < 1e-13  # F_eta, T_eta: rounding of ~10^3 link terms
    assert np.abs(P[6:12]).max() == 0.0  # no interface: no capillary force


def test_momentum_exchange_balances_fluid_momentum():
    """Fixed sphere in a body-force driven flow: the fluid momentum changes per step
    by N_fluid g - F_eta exactly (momentum exchange = momentum the links remove)."""
    n, g = 18, 2e-5
    s = O.OracleSim(n, n, n, body_force_a=(g, 0.5 * g, 0.0), body_force_b=(g, 0.5 * g, 0.0), sigma=0.0)
    s.init_fields(np.ones(n ** 3))
    s.add_particle((8.3, 9.1, 8.6), 4.4, kinematic=True)
    nfluid = int((s.owner() == 0).sum())
    s.step(30)
    P0 = s.diag()[4:7]
    for _ in range(5):
        s.step(1)
        P1 = s.diag()[4:7]
        Feta = s.particles()[0][0:3]
        expect = nfluid * np.array([g, 0.5 * g, 0.0]) - Feta
        assert np.abs((P1 - P0) - expect).max() < 1e-12 * max(1.0, np.abs(Feta).max())
        assert np.abs(Feta).max() > 1e-4  # the flow does load the sphere
        P0 = P1


def test_moving_sphere_mass_bookkeeping():
    """Kinematic sphere crossing nodes: total mass changes by bounce-back source +
    refilled mass - covered mass, step by step (Sec. V A, V C)."""
    n = 20
    s = O.OracleSim(n, n, n, sigma=0.0)
    s.init_fields(np.ones(n ** 3))
    s.add_particle((6.2, 10.0, 10.0), 3.7, v=(0.21, 0.07, 0.0), kinematic=True)
    s.step(1)
    M0 = s.diag()[3]
    seen_refill = seen_cover = False
    for _ in range(25):
        s.step(1)
        d = s.diag()
        assert abs(d[3] - (M0 + d[0] + d[1] - d[2])) < 1e-12 * M0
        seen_refill |= d[1] > 0
        seen_cover |= d[2] > 0
        M0 = d[3]
    assert seen_refill and seen_cover


def test_capillary_symmetric_interface_zero_force():
    """Sphere centred on a flat interface, 90 deg: the force cancels by symmetry."""
    n = 33
    z = np.arange(n, dtype=float)
    phi = np.broadcast_to(np.tanh(0.5 * (z - 16.0))[:, None, None], (n, n, n)).reshape(-1)
    s = O.OracleSim(n, n, n, sigma=0.01)
    s.init_fields(phi)
    s.add_particle((16.0, 16.0, 16.0), 8.0, theta_deg=90.0, kinematic=True)
    s.eval_interface()
    F, T, used = s.capillary(0)
    assert used > 0
    scale = 0.01 * 8.0
    assert np.abs(F).max() < 1e-12 * scale
    assert np.abs(T).max() < 1e-12 * scale * 8.0


def test_capillary_matches_surface_integral():
    """Sec. V E: the Lagrangian-point sum approximates
    C sigma oint (1 - phi^2) [n_s - (n.n_s) n] dA over the sphere, evaluated here by
    brute-force quadrature of the analytic field of a spherical drop crossing the
    particle (wetting rotation disabled so the gradient is the plain stencil)."""
    n, a, Rd, Rp, sigma, C = 48, 0.5, 14.0, 10.0, 0.01, 1.0
    xd = np.array([n / 2, n / 2, n / 2 - 5.0])
    xp = np.array([n / 2, n / 2, n / 2 - 5.0 + Rd + 0.3 * Rp])
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    r = np.sqrt((x - xd[0]) ** 2 + (y - xd[1]) ** 2 + (z - xd[2]) ** 2)
    s = O.OracleSim(n, n, n, sigma=sigma, cap_norm=C, wet_phi_max=0.0)
    s.init_fields(np.tanh(a * (Rd - r)).reshape(-1))
    s.add_particle(xp, Rp, kinematic=True)
    s.eval_interface()
    F, T, _ = s.capillary(0)
    na = nv = 720
    al = (np.arange(na) + 0.5) * math.pi / na
    vp = np.arange(nv) * 2 * math.pi / nv
    A, V = np.meshgrid(al, vp, indexing="ij")
    ns = np.stack([np.sin(A) * np.cos(V), np.sin(A) * np.sin(V), np.cos(A)], -1)
    d = xp + Rp * ns - xd
    rr = np.linalg.norm(d, axis=-1)
    ph = np.tanh(a * (Rd - rr))
    nh = -d / rr[..., None]
    m = ns - (nh * ns).sum(-1)[..., None] * nh
    dA = Rp ** 2 * np.sin(A) * (math.pi / na) * (2 * math.pi / nv)
    Fb = ((C * sigma * (1 - ph ** 2) * dA)[..., None] * m).sum((0, 1))
    assert Fb[2] < 0  # the drop below pulls the particle down along the line of centres
    assert abs(F[2] / Fb[2] - 1) < 0.05
    assert np.abs(F[:2]).max() < 1e-12 and np.abs(T).max() < 1e-12
