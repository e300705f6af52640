"""Flow-level pins of the oracle: channel flow, moving wall, mass conservation."""
import numpy as np

import oracle as O
from paper_2505_10171_gb300 import workloads as W


def test_poiseuille_between_halfway_walls_is_exact():
    """Body-force channel between halfway bounce-back walls at z=0.5 and z=nz-0.5:
    with the Lambda = 3/16 rates the steady profile is the exact parabola
    u(z) = g (z - z0)(z1 - z)/(2 nu)."""
    nz, g = 12, 1e-6
    for nu in (1.0 / 6.0, 0.05):
        s = O.OracleSim(1, 1, nz, wall_z0=1, nu_a=nu, nu_b=nu, body_force_a=(g, 0, 0), body_force_b=(g, 0, 0))
        s.init_fields(np.ones(nz))
        s.step(int(6.0 * nz * nz / nu))
        u = s.fields()["u"][0]
        z = np.arange(nz)
        ua = g * (z - 0.5) * (nz - 0.5 - z) / (2 * nu)
        ua[0] = 0.0
        assert np.abs(u - ua).max() / ua.max() < 1e-9


def test_uniform_flow_over_moving_wall_is_steady():
    """f = feq(rho, U) with the substrate moving at U is an exact fixed point of
    streaming + moving bounce-back + collision."""
    nx, ny, nz = 6, 5, 7
    U = (2e-3, -1e-3, 0.0)
    s = O.OracleSim(nx, ny, nz, wall_z0=1, wall_velocity=U)
    u = np.zeros((3, nx * ny * nz))
    u[0], u[1] = U[0], U[1]
    s.init_fields(np.ones(nx * ny * nz), u=u)
    fa0, _ = s.pops()
    s.step(20)
    fa1, _ = s.pops()
    assert np.abs(fa1 - fa0).max() < 1e-15
    uu = s.fields()["u"].reshape(3, nz, ny, nx)[:, 1:]
    assert np.abs(uu[0] - U[0]).max() < 1e-15 and np.abs(uu[1] - U[1]).max() < 1e-15


def test_component_mass_conserved_drop_on_sliding_wall():
    """Recolouring keeps rho^a and rho^b per node; tangential wall motion adds no
    mass per node (sum_i w_i c_i.u_w over the wall links is zero)."""
    nx, ny, nz = 24, 16, 14
    phi = W.drop_phi(nx, ny, nz, (10.0, 8.0, 0.5), 6.0)
    s = O.OracleSim(nx, ny, nz, wall_z0=1, wall_velocity=(1e-3, 0, 0), theta_wall_deg=70.0,
                    nu_b=1.0 / 30.0, sigma=0.02)
    s.init_fields(phi)
    f0 = s.fields()
    ma0, mb0 = f0["rho_a"].sum(), f0["rho_b"].sum()
    s.step(200)
    f1 = s.fields()
    assert abs(f1["rho_a"].sum() - ma0) / ma0 < 1e-13
    assert abs(f1["rho_b"].sum() - mb0) / mb0 < 1e-13
    assert np.isfinite(f1["u"]).all()


def test_drop_speed_controller_follows_the_pi_recurrence():
    """Reading c27: PI control of the phase-a body force.  In a uniform
    single-phase periodic box Guo forcing adds exactly f to the momentum per
    node and step, so the measured velocity after step t is U(t) = U(t-1) +
    f(t)/rho0 and the force follows the PI law updated every `iv` steps; the
    oracle must reproduce that scalar recurrence."""
    n, iv, kp, ki, target, f0 = 6, 10, 2e-2, 1e-4, 1e-3, 2e-6
    # run the oracle in pieces that straddle update points
    s2 = O.OracleSim(n, n, n, body_force_a=(f0, 0.0, 0.0), drop_speed_control=1,
                     drop_speed_target=(target, 0.0, 0.0), drop_speed_kp=kp, drop_speed_ki=ki,
                     drop_speed_interval=iv)
    s2.init_fields(np.ones(n ** 3))
    U, f, integ, t, Ulast = 0.0, f0, 0.0, 0, 0.0
    for chunk in (7, 3, 45, 145):
        s2.step(chunk)
        for _ in range(chunk):
            t += 1
            U += f
            if t % iv == 0:
                Ulast = U
                e = target - U
                integ += e * iv
                f = f0 + kp * e + ki * integ
        force, uref = s2.speed_control()
        # the measured velocity is a momentum formed from O(0.1) populations:
        # compare to absolute round-off
        assert abs(uref[0] - Ulast) <= 1e-13
        assert abs(force[0] - f) <= 1e-15
        assert force[1] == 0.0 and force[2] == 0.0
    # the controlled run approaches the target
    assert abs(U - target) < 0.5 * target
