"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it only draws initial fields
(order parameter, density, velocity), static solid masks and particle lists.
Both the CUDA path and the CPU oracle are fed from it.  Every array is
z-major (index = (z*ny + y)*nx + x) and FP64.

The shapes follow the paper's own set-ups (Sec. VI A: a hemispherical drop on
a flat substrate with a sphere in front of it, periodic in x, y, z; Table I
parameter ranges; Sec. V D: Segre-Silberberg tube), with the sizes of the
configurations this library is measured on:

* ``cfg1`` - 48x32x32, drop R=10, one sphere R_p=4, 200 steps (parity case).
* ``cfg2`` - 256x128x128, drop R=40, eight spheres R_p=8, 20000 steps.
* ``cfg3`` - 64x64x1024 tube R_t=31, single phase, one sphere R_p=6.
* ``cfg4`` - 96 independent drop/sphere instances of uneven size.
"""
from __future__ import annotations

import math

import numpy as np

# Table I (simulation units) and the common defaults of the configurations.
COMMON = dict(
    rho0=1.0, beta=0.7, sigma=0.01, delta_R=1.0,
    kn=2.5, kt=1.0, kr=0.5, gn=0.0, gt=0.0, gr=0.0,
)
INTERFACE_WIDTH = 2.5
# Table I: particle density 0.125 against fluid density 0.05, i.e. a particle
# 2.5 times denser than the fluid; with rho0 = 1 the particle density is 2.5.
PARTICLE_DENSITY = 2.5


def grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)


def periodic_delta(d, n):
    """Minimum-image displacement on a periodic axis of n nodes."""
    return d - n * np.floor(d / n + 0.5)


def drop_phi(nx, ny, nz, centre, R, width=INTERFACE_WIDTH):
    """Order parameter of a spherical drop: +1 inside, -1 outside, tanh edge."""
    x, y, z = grid(nx, ny, nz)
    dx = periodic_delta(x - centre[0], nx)
    dy = periodic_delta(y - centre[1], ny)
    dz = periodic_delta(z - centre[2], nz)
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    return np.tanh(2.0 * (R - r) / width).reshape(-1)


def cfg1():
    """48x32x32 parity case: drop R=10 on a wall sliding at 1e-3, sphere R_p=4."""
    nx, ny, nz = 48, 32, 32
    params = dict(COMMON, nx=nx, ny=ny, nz=nz, wall_z0=1, wall_velocity=(1e-3, 0.0, 0.0),
                  theta_wall_deg=90.0, nu_a=1.0 / 6.0, nu_b=1.0 / 6.0, mu_s=0.3, mu_r=0.05,
                  g_particle=(0.0, 0.0, 0.0))
    phi = drop_phi(nx, ny, nz, (16.0, 16.0, 0.5), 10.0)
    particles = [dict(x=(33.0, 16.0, 5.5), R=4.0, rho_p=PARTICLE_DENSITY, theta_deg=60.0)]
    return dict(name="drop-sphere 48x32x32, 1 sphere R=4, FP64 parity", params=params, phi=phi,
                particles=particles, steps=200)


def place_spheres(rng, n, R, Rc, x_range, y_range, z, min_spacing, max_tries=100000):
    """Rejection-sample n non-overlapping sphere centres at height z."""
    out = []
    tries = 0
    while len(out) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place spheres")
        x = rng.uniform(*x_range)
        y = rng.uniform(*y_range)
        if all((x - a) ** 2 + (y - b) ** 2 >= min_spacing ** 2 for a, b, _ in out):
            out.append((x, y, z))
    return out


def resting_damping(R_p, rho_p=PARTICLE_DENSITY):
    """Normal contact damping at half the critical value for a sphere resting
    on the wall.  Undamped, a sphere released at first contact overshoots its
    rest overlap by as much again; with the weight 10 sigma R_p and k_n = 2.5 an
    R_p = 8 sphere then covers the fluid nodes between itself and the wall,
    and the momentum exchange on its open surface (the rest pressure on the
    top, none underneath) pushes it into the substrate."""
    m = rho_p * 4.0 / 3.0 * math.pi * R_p ** 3
    return 0.5 * 2.0 * math.sqrt(COMMON["kn"] * m)


def cfg2(seed=20251, n_spheres=8):
    """256x128x128 resolved run: drop R=40 driven along x over a 150 deg wall
    (body force on the drop, PI-controlled every 100 steps towards a drop speed
    of 5e-3), eight spheres R_p=8 with contact angles uniform in [30, 90] deg,
    drop:ambient kinematic viscosities 1/6 : 1/60, normal contact damping at
    half the critical value."""
    nx, ny, nz = 256, 128, 128
    R_p, Rc = 8.0, 9.0
    rng = np.random.default_rng(seed)
    centres = place_spheres(rng, n_spheres, R_p, Rc, (96 + Rc + 4, nx - Rc - 4), (Rc, ny - Rc),
                            9.5, 2 * Rc + 1)
    thetas = rng.uniform(30.0, 90.0, size=n_spheres)
    sigma = COMMON["sigma"]
    params = dict(COMMON, nx=nx, ny=ny, nz=nz, wall_z0=1, wall_velocity=(0.0, 0.0, 0.0),
                  theta_wall_deg=150.0, nu_a=1.0 / 6.0, nu_b=1.0 / 60.0, mu_s=0.3, mu_r=0.05,
                  gn=resting_damping(R_p),
                  body_force_a=(2.0e-6, 0.0, 0.0), g_particle=(0.0, 0.0, -10.0 * sigma * R_p),
                  drop_speed_control=1, drop_speed_target=(5.0e-3, 0.0, 0.0), drop_speed_interval=100)
    phi = drop_phi(nx, ny, nz, (48.0, 64.0, 0.5), 40.0)
    particles = [dict(x=c, R=R_p, rho_p=PARTICLE_DENSITY, theta_deg=float(t)) for c, t in zip(centres, thetas)]
    return dict(name="drop-sphere 256x128x128, 8 spheres R=8", params=params, phi=phi,
                particles=particles, steps=20000)


def cfg3(nz=1024):
    """64x64xnz tube of radius 31 (periodic along z), single phase, body-force
    driven Poiseuille flow at centreline speed 0.02, one neutrally buoyant
    sphere R_p=6 released at r = 0.3 R_t."""
    nx = ny = 64
    Rt, uc, nu = 31.0, 0.02, 1.0 / 6.0
    x, y, z = grid(nx, ny, nz)
    r = np.sqrt((x - 31.5) ** 2 + (y - 31.5) ** 2).reshape(-1)
    mask = (r > Rt).astype(np.uint8)
    g = 4.0 * nu * uc / Rt ** 2
    u = np.zeros((3, nx * ny * nz))
    u[2] = np.where(r <= Rt, uc * (1.0 - (r / Rt) ** 2), 0.0)
    l = 0.3 * Rt
    params = dict(COMMON, nx=nx, ny=ny, nz=nz, wall_z0=0, nu_a=nu, nu_b=nu, sigma=0.0,
                  body_force_a=(0.0, 0.0, g), mu_s=0.0, mu_r=0.0)
    up = uc * (1.0 - (l / Rt) ** 2)
    particles = [dict(x=(31.5 + l, 31.5, nz / 2), R=6.0, rho_p=1.0, theta_deg=90.0, v=(0.0, 0.0, up))]
    return dict(name=f"tube 64x64x{nz}, sphere R=6", params=params, phi=np.ones(nx * ny * nz), u=u,
                mask=mask, particles=particles, steps=50000)


# the anti-bounce-back faces realise an imposed density drop about this many
# lattice units inside each face (measured on a pressure-driven channel)
FACE_SHIFT = 1.6


def tube_pressure(R_t=40.0, R_p=12.2, nz=2560, rho=1.05, nu=0.457, v_in=0.0113, l0=0.21, z0=200.0):
    """Segre-Silberberg tube of Sec. V D at the paper's parameters: tube of
    radius R_t along z, pressure faces at both ends (anti-bounce-back) with
    the density drop of Poiseuille flow at mean speed v_in over the effective
    length, single phase of density rho and viscosity nu, a neutrally buoyant
    sphere R_p released at l0 R_t from the axis with the local flow speed.
    The initial flow is the Poiseuille profile."""
    nx = ny = int(2 * R_t) + 2
    c = (nx - 1) / 2.0
    x, y, z = grid(nx, ny, nz)
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2).reshape(-1)
    mask = (r > R_t).astype(np.uint8)
    L_eff = nz - 2 - 2 * FACE_SHIFT
    drho = 3.0 * 8.0 * rho * nu * v_in / R_t ** 2 * L_eff
    u = np.zeros((3, nx * ny * nz))
    u[2] = np.where(r <= R_t, 2.0 * v_in * (1.0 - (r / R_t) ** 2), 0.0)
    params = dict(COMMON, nx=nx, ny=ny, nz=nz, wall_z0=0, rho0=rho, nu_a=nu, nu_b=nu, sigma=0.0,
                  pressure_z=1, rho_in=rho + drho / 2, rho_out=rho - drho / 2, mu_s=0.0, mu_r=0.0)
    l = l0 * R_t
    up = 2.0 * v_in * (1.0 - (l / R_t) ** 2)
    particles = [dict(x=(c + l, c, z0), R=R_p, rho_p=rho, theta_deg=90.0, v=(0.0, 0.0, up))]
    return dict(name=f"pressure-driven tube R_t={R_t:g}, sphere R_p={R_p:g}, {nx}x{ny}x{nz}", params=params,
                phi=np.ones(nx * ny * nz), rho=np.full(nx * ny * nz, rho), u=u, mask=mask, particles=particles,
                R_t=R_t, centre=c)


def capture_case(mu, mu_r, scale=0.5, Bo=1.25, friction_number=5.23, sigma=0.01, offset=0.5):
    """One drop-particle collision of the friction map of Sec. VI C, its
    shapes scaled by `scale` from the paper's (400x181x71 lattice, R_p = 10,
    R_d = 5 R_p): a hemispherical drop (phase a) on the substrate, pushed
    along x by the force density f_x = Bo sigma / R_d^2 on phase a (the
    printed Bo = f_x R_d / sigma is not dimensionless for a force per unit
    volume; with R_d^2 and sigma = 0.01 the total force on the R_d = 50 drop
    is 1.3, inside Table I's 0.26 - 1.57), and a sphere
    resting on the substrate ahead of it, `offset` R_p to the side, weight
    g_p = friction_number sigma R_p (so that mu g_p/(sigma R_p) spans 0 to
    friction_number as mu goes from 0 to 1), contact angles 90 deg on sphere
    and substrate, sliding / rolling friction mu, mu_r.  Viscosities of the
    256x128x128 run (drop 1/6, ambient 1/60), particle density of the
    workloads, normal contact damping at half the critical value."""
    nx, ny, nz = int(round(400 * scale)), int(round(181 * scale)), int(round(71 * scale))
    R_p = 10.0 * scale
    R_d = 5.0 * R_p
    f_x = Bo * sigma / R_d ** 2
    g_p = friction_number * sigma * R_p
    xd = 1.0 + R_d + 6.0 * scale
    params = dict(COMMON, nx=nx, ny=ny, nz=nz, wall_z0=1, theta_wall_deg=90.0, sigma=sigma, nu_a=1.0 / 6.0,
                  nu_b=1.0 / 60.0, body_force_a=(f_x, 0.0, 0.0), mu_s=mu, mu_r=mu_r, gn=resting_damping(R_p),
                  g_particle=(0.0, 0.0, -g_p))
    phi = drop_phi(nx, ny, nz, (xd, ny / 2.0, 0.5), R_d)
    zc = 0.5 + R_p + params["delta_R"] - g_p / params["kn"]
    particles = [dict(x=(xd + R_d + R_p + 3.0, ny / 2.0 + offset * R_p, zc), R=R_p, rho_p=PARTICLE_DENSITY,
                      theta_deg=90.0)]
    return dict(name=f"capture case mu={mu:g} mu_r={mu_r:g}", params=params, phi=phi, particles=particles,
                R_d=R_d, Bo=Bo)


def ceil8(v):
    return int(math.ceil(v / 8.0) * 8)


def cfg4(seed=4242, n_instances=96):
    """Batched sweep: drop radius uniform in [16, 40], domain 5.5R x 3.2R x 3.2R
    rounded up to multiples of 8 (at least 96x64x64), one sphere R/5, drop speed
    uniform in [1e-3, 1e-2], mu_s in [0, 0.6], mu_r in [0, 0.1]."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_instances):
        Rd = rng.uniform(16.0, 40.0)
        U = rng.uniform(1e-3, 1e-2)
        mu_s = rng.uniform(0.0, 0.6)
        mu_r = rng.uniform(0.0, 0.1)
        nx, ny, nz = max(96, ceil8(5.5 * Rd)), max(64, ceil8(3.2 * Rd)), max(64, ceil8(3.2 * Rd))
        R_p = Rd / 5.0
        sigma = COMMON["sigma"]
        params = dict(COMMON, nx=nx, ny=ny, nz=nz, wall_z0=1, theta_wall_deg=90.0,
                      nu_a=1.0 / 6.0, nu_b=1.0 / 60.0, mu_s=mu_s, mu_r=mu_r, gn=resting_damping(R_p),
                      body_force_a=(U * 4e-4, 0.0, 0.0), g_particle=(0.0, 0.0, -10.0 * sigma * R_p),
                      drop_speed_control=1, drop_speed_target=(U, 0.0, 0.0), drop_speed_interval=100)
        xd = 1.2 * Rd
        phi = drop_phi(nx, ny, nz, (xd, ny / 2.0, 0.5), Rd)
        xp = xd + Rd + R_p + 3.0
        particles = [dict(x=(xp, ny / 2.0, R_p + 1.5), R=R_p, rho_p=PARTICLE_DENSITY, theta_deg=90.0)]
        out.append(dict(params=params, phi=phi, particles=particles, drop_speed=U))
    return out


def cfg2_crop(nx=64, ny=64, nz=32, seed=20251, sphere=5):
    """A sub-box of the 256x128x128 resolved run (same parameters and fields,
    cut out around one of its spheres, the one nearest the drop by default),
    for bounded CPU samples of that workload."""
    full = cfg2(seed)
    N0 = (256, 128, 128)
    p0 = full["particles"][sphere]["x"]
    x0 = int(p0[0]) - nx // 2
    y0 = int(p0[1]) - ny // 2
    params = dict(full["params"], nx=nx, ny=ny, nz=nz)
    x, y, z = grid(nx, ny, nz)
    dx = periodic_delta(x + x0 - 48.0, N0[0])
    dy = periodic_delta(y + y0 - 64.0, N0[1])
    dz = z - 0.5
    phi = np.tanh(2.0 * (40.0 - np.sqrt(dx * dx + dy * dy + dz * dz)) / INTERFACE_WIDTH).reshape(-1)
    parts = []
    for q in full["particles"]:
        xx, yy, zz = q["x"][0] - x0, q["x"][1] - y0, q["x"][2]
        R = q["R"] + 2.0
        if R <= xx < nx - R and R <= yy < ny - R and zz + R < nz - 1:
            parts.append(dict(q, x=(xx, yy, zz)))
    return dict(name=f"sub-box {nx}x{ny}x{nz} of the 256x128x128 run", params=params, phi=phi, particles=parts)
