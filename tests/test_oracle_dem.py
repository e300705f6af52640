"""Pins of the oracle's DEM (Sec. III): bounce, restitution, incline, rolling."""
import json
import math
import os

import numpy as np

import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
T1 = GOLD["table1_dem"]
R = T1["R_p"]
RHO_P = T1["rho_p"]
M = RHO_P * 4.0 / 3.0 * math.pi * R ** 3


def test_collision_time_matches_paper_step_ratio():
    """Sec. V H: t_c = pi/omega_c, omega_c = sqrt(k_n/m - (g_n/2m)^2); with the
    Table I values and m from R_p, Delta t = 1 ~ t_c/45."""
    tc = math.pi / math.sqrt(T1["kn"] / M)
    g = GOLD["dt_over_tc"]
    assert abs(tc / g["value"] - 1) < g["tol_rel"]


def apexes(z):
    return [z[i] for i in range(1, len(z) - 1) if z[i] >= z[i - 1] and z[i] > z[i + 1] and z[i] > 0.5]


def bounce(gn, steps=60000, g=1e-5, h0=40.0):
    s = O.OracleSim(8, 8, 400, wall_z0=1, kn=T1["kn"], gn=gn, delta_R=0.0, g_particle=(0, 0, -M * g))
    s.add_particle((4, 4, 0.5 + R + h0), R, rho_p=RHO_P)
    tr = s.dem_only(steps)
    return tr, tr[:, 0, 2] - 0.5 - R, g, h0


def test_elastic_bounce_keeps_apex_and_energy():
    tr, z, g, h0 = bounce(0.0)
    ap = apexes(z)
    assert len(ap) >= 5
    assert max(abs(a / h0 - 1) for a in ap[:5]) < 3e-3
    # free-flight segment follows h(t) = h0 - g t^2/2 before the first impact
    t = np.arange(1, 1000)
    assert np.abs(z[t - 1] - (h0 - 0.5 * g * t ** 2)).max() < 1e-9
    E = 0.5 * M * (tr[:, 0, 3:6] ** 2).sum(1) + M * g * z
    flight = z > 1.0
    assert np.abs(E[flight] / (M * g * h0) - 1).max() < 1e-2  # bounded, no secular drift


def test_damped_bounce_restitution():
    """h_n = r^(2n) h_0 with r = exp(-eta_n t_c), eta_n = g_n/(2m) (the printed
    exp(eta_n/t_c) would give no visible decay)."""
    gn = GOLD["bounce_incline"]["gamma_n_damped"]
    _, z, _, h0 = bounce(gn)
    eta = gn / (2 * M)
    tc = math.pi / math.sqrt(T1["kn"] / M - eta ** 2)
    r = math.exp(-eta * tc)
    ap = apexes(z)
    for k in range(4):
        assert abs(ap[k] / h0 / r ** (2 * (k + 1)) - 1) < 1e-2


def incline(mu_s, mu_r, steps=20000, g=2e-5):
    th = math.radians(GOLD["bounce_incline"]["incline_deg"])
    gvec = (M * g * math.sin(th), 0, -M * g * math.cos(th))
    s = O.OracleSim(400, 8, 64, wall_z0=1, kn=T1["kn"], kt=T1["kt"], kr=T1["kr"], mu_s=mu_s, mu_r=mu_r,
                    delta_R=0.0, g_particle=gvec)
    s.add_particle((20, 4, 0.5 + R - M * g * math.cos(th) / T1["kn"]), R, rho_p=RHO_P)
    return s.dem_only(steps), g, th


def test_frictionless_incline_slides_without_rotation():
    tr, g, th = incline(0.0, 0.0)
    assert np.abs(tr[:, 0, 6:9]).max() == 0.0
    v = tr[:, 0, 3]
    a = (v[-1] - v[-5001]) / 5000
    assert abs(a / (g * math.sin(th)) - 1) < 1e-10


def test_frictional_incline_rolls_with_small_slip():
    """mu > (2/7) tan(theta): rolling without slip, a = (5/7) g sin(theta),
    |s| ~ 1e-3 (Sec. III D)."""
    tr, g, th = incline(0.5, 0.0)
    v, w = tr[:, 0, 3], tr[:, 0, 7]
    a = (v[-1] - v[-5001]) / 5000
    assert abs(a / (5 / 7 * g * math.sin(th)) - 1) < 1e-3
    s = w[-1] * R / v[-1] - 1
    gs = GOLD["slip_ratio_abs"]
    assert abs(abs(s) - gs["value"]) <= gs["tol_abs"]
    assert w[-1] > 0  # rolls down the slope (about +y for motion along +x)


def test_rolling_friction_slows_rolling():
    """With mu_r > 0: a = (5/7) g (sin theta - mu_r cos theta) (R_c = R_p here)."""
    mu_r = 0.05
    tr, g, th = incline(0.5, mu_r)
    v = tr[:, 0, 3]
    a = (v[-1] - v[-5001]) / 5000
    assert abs(a / (5 / 7 * g * (math.sin(th) - mu_r * math.cos(th))) - 1) < 2e-3


def test_rolling_marker_traces_cycloid():
    """Sec. III D, Eq. (cycloid): a surface marker of a rolling sphere follows
    x = R(alpha - sin alpha), z = R(1 - cos alpha) + z0 relative to its start."""
    tr, g, th = incline(0.5, 0.0, steps=6000)
    x = tr[:, 0, 0]
    q = tr[:, 0, 9:13]
    # marker initially at the contact point: body vector (0, 0, -R)
    def rot(qq, v):
        w_, x_, y_, z_ = qq
        Rm = np.array([[1 - 2 * (y_ * y_ + z_ * z_), 2 * (x_ * y_ - w_ * z_), 2 * (x_ * z_ + w_ * y_)],
                       [2 * (x_ * y_ + w_ * z_), 1 - 2 * (x_ * x_ + z_ * z_), 2 * (y_ * z_ - w_ * x_)],
                       [2 * (x_ * z_ - w_ * y_), 2 * (y_ * z_ + w_ * x_), 1 - 2 * (x_ * x_ + y_ * y_)]])
        return Rm @ v
    err = 0.0
    x0 = x[0]
    for k in range(0, len(x), 50):
        m = rot(q[k], np.array([0.0, 0.0, -R]))
        mx, mz = x[k] + m[0] - x0, R + m[2]
        alpha = (x[k] - x0) / R
        err = max(err, abs(mx - R * (alpha - math.sin(alpha))), abs(mz - R * (1 - math.cos(alpha))))
    assert x[-1] - x0 > 2 * math.pi * R  # at least one full turn
    assert err < 0.02 * R


def test_head_on_pair_collision_exchanges_velocity():
    """Two equal spheres, elastic normal contact: momentum conserved, velocities swap."""
    s = O.OracleSim(200, 40, 40, kn=T1["kn"], delta_R=1.0)
    s.add_particle((60.0, 20.0, 20.0), R, rho_p=RHO_P, v=(0.01, 0, 0))
    s.add_particle((90.0, 20.0, 20.0), R, rho_p=RHO_P, v=(0.0, 0, 0))
    tr = s.dem_only(3000)
    v1, v2 = tr[-1, 0, 3], tr[-1, 1, 3]
    assert abs((v1 + v2) - 0.01) < 1e-15
    assert abs(v1) < 2e-4 and abs(v2 - 0.01) < 2e-4
