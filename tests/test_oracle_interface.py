"""Interface pins of the oracle: recolouring profile, CSF/Laplace, wetting (Sec. IV, V E)."""
import json
import math
import os

import numpy as np

import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
K = (1 + math.sqrt(2)) / 18


def planar(beta, steps=4000, nx=64):
    x = np.arange(nx)
    phi = np.where((x >= nx // 4) & (x < 3 * nx // 4), 1.0, -1.0)
    s = O.OracleSim(nx, 1, 1, beta=beta, sigma=0.0, grad_eps=1e-14)  # unregularised limit
    s.init_fields(phi)
    s.step(steps)
    return s.fields()["phi"]


def test_planar_interface_integral_and_profile():
    """At rest, a planar interface settles where, for every x,
    (phi(x+1) - phi(x))/6 = beta k [1 - (phi(x+1)^2 + phi(x)^2)/2], hence
    sum_x (1 - phi^2) = 1/(3 k beta) across one interface; this is the quantity
    the capillary prefactor of Sec. V F is built on."""
    for beta in (0.7, 0.99):
        ph = planar(beta)
        half = len(ph) // 2
        s1 = (1 - ph[:half] ** 2).sum()
        s2 = (1 - ph[half:] ** 2).sum()
        assert abs(s1 - 1 / (3 * K * beta)) < 1e-7
        assert abs(s2 - 1 / (3 * K * beta)) < 1e-7
        nxt = np.roll(ph, -1)
        res = (nxt - ph) / 6 - beta * K * np.sign(nxt - ph) * (1 - (nxt ** 2 + ph ** 2) / 2)
        assert np.abs(res).max() < 1e-8
        # monotone, tanh-like, symmetric profile
        i0 = np.argmin(np.abs(ph[:half]))
        assert np.all(np.diff(ph[i0 - 4:i0 + 5]) > 0)


def test_laplace_law_cylinder_converges():
    """Sec. IV CSF: a static cylindrical drop (one periodic node along z) carries
    p_in - p_out = sigma/R; the error shrinks with R (diffuse interface)."""
    n, sigma = 64, 0.01
    X, Y = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    errs = []
    for R in (8, 16):
        rr = np.sqrt((X - 31.5) ** 2 + (Y - 31.5) ** 2)
        s = O.OracleSim(n, n, 1, sigma=sigma)
        s.init_fields(np.tanh(2 * (R - rr) / 2.5).reshape(-1))
        s.step(3000)
        f = s.fields()
        rho = (f["rho_a"] + f["rho_b"]).reshape(n, n)
        ph = f["phi"].reshape(n, n)
        dp = rho[28:36, 28:36].mean() / 3 - rho[:4, :4].mean() / 3
        Req = math.sqrt(((ph + 1) / 2).sum() / math.pi)
        assert dp > 0  # inward CSF force: higher pressure inside the phi=+1 drop
        errs.append(abs(dp / (sigma / Req) - 1))
    assert errs[1] < errs[0]
    assert errs[1] < 0.03


def test_laplace_law_sphere():
    """3-D drop: p_in - p_out = 2 sigma/R (two principal curvatures)."""
    n, sigma, R = 36, 0.01, 9
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    rr = np.sqrt((x - 17.5) ** 2 + (y - 17.5) ** 2 + (z - 17.5) ** 2)
    s = O.OracleSim(n, n, n, sigma=sigma)
    s.init_fields(np.tanh(2 * (R - rr) / 2.5).reshape(-1))
    s.step(1200)
    f = s.fields()
    rho = (f["rho_a"] + f["rho_b"]).reshape(n, n, n)
    ph = f["phi"].reshape(n, n, n)
    dp = rho[15:21, 15:21, 15:21].mean() / 3 - rho[:3, :3, :3].mean() / 3
    Req = (3 * ((ph + 1) / 2).sum() / (4 * math.pi)) ** (1 / 3)
    assert abs(dp / (2 * sigma / Req) - 1) < 0.08


def test_wetting_rotation_properties():
    """Sec. V E: the rotated gradient keeps |grad phi|; its direction -n makes the
    prescribed angle with n_s; of n_+ and n_- the one closer to n* is taken."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        g = rng.normal(size=3)
        ns = rng.normal(size=3)
        ns /= np.linalg.norm(ns)
        th = rng.uniform(0.2, math.pi - 0.2)
        g2 = O.wetting_rotate(g, ns, th)
        assert abs(np.linalg.norm(g2) - np.linalg.norm(g)) < 1e-13
        n_new = -g2 / np.linalg.norm(g2)
        assert abs(n_new @ ns - math.cos(th)) < 1e-12
        nstar = -g / np.linalg.norm(g)
        # n_new lies in the plane of n_s and n*, on the side of n*
        assert abs(np.linalg.det(np.stack([n_new, ns, nstar]))) < 1e-12
        other = 2 * (ns @ n_new) * ns - n_new  # the mirror candidate about n_s
        assert n_new @ nstar >= other @ nstar - 1e-12


def fit_cap_angle(ph, nx, nz, zmin=3):
    pts = []
    for z in range(zmin, nz - 1):
        row = ph[z]
        for x in range(nx - 1):
            if row[x] * row[x + 1] < 0:
                pts.append((x + row[x] / (row[x] - row[x + 1]), z))
    for x in range(nx):
        col = ph[:, x]
        for z in range(zmin, nz - 1):
            if col[z] * col[z + 1] < 0:
                pts.append((x, z + col[z] / (col[z] - col[z + 1])))
    P = np.array(pts)
    A = np.c_[2 * P[:, 0], 2 * P[:, 1], np.ones(len(P))]
    xc, zc, c = np.linalg.lstsq(A, (P ** 2).sum(1), rcond=None)[0]
    return math.degrees(math.acos((0.5 - zc) / math.sqrt(c + xc ** 2 + zc ** 2)))


def test_sessile_contact_angle():
    """A 2-D sessile drop relaxes to the prescribed angle, measured inside phase a,
    within the paper's stated accuracy (~6%, worst ~16%, Sec. V E)."""
    nx, nz, R = 72, 28, 11
    X, Z = np.meshgrid(np.arange(nx), np.arange(nz), indexing="xy")
    phi = np.tanh(2 * (R - np.sqrt((X - 36) ** 2 + (Z - 0.5) ** 2)) / 2.5)
    gold = GOLD["wetting_error_rel"]
    meas = {}
    for th in (60.0, 90.0, 120.0):
        s = O.OracleSim(nx, 1, nz, wall_z0=1, theta_wall_deg=th, sigma=0.01)
        s.init_fields(phi.reshape(-1))
        s.step(6000)
        meas[th] = fit_cap_angle(s.fields()["phi"].reshape(nz, nx), nx, nz)
        assert abs(meas[th] - th) / th < gold["worst"]
    assert abs(meas[120.0] - 120.0) / 120.0 < gold["typical"]
    assert abs(meas[90.0] - 90.0) / 90.0 < gold["typical"]
    assert meas[60.0] < meas[90.0] < meas[120.0]


def test_default_capillary_prefactor_gives_sigma_per_unit_line():
    """The default prefactor C = 3 k beta turns the settled planar profile's
    sum (1 - phi^2) into exactly one: a straight contact line of length L
    across the interface carries sigma L (the line-integral form of Sec. V F);
    the printed (9/2) k beta would carry 1.5 sigma L."""
    for beta in (0.7, 0.99):
        ph = planar(beta)
        s1 = (1 - ph[:len(ph) // 2] ** 2).sum()
        C = O.make_params(8, 8, 8, beta=beta).cap_norm
        assert abs(C * s1 - 1.0) < 1e-7
        assert abs(4.5 * K * beta * s1 - 1.5) < 1e-7
