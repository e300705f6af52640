"""Benchmarks of the method against closed forms, run through the C ABI.

Capillary detachment (Sec. V G, benchmarking the capillary force; Scheludko's maximum force): a sphere held at
its equilibrium height in a flat interface is pulled out at constant speed, and
the largest capillary force opposing the motion is compared with
F_max = 2 pi sigma R_p cos^2(theta_p / 2).

Wetting equilibrium (Sec. V E, wetting boundary condition: the particle-at-interface benchmark): a free
sphere released halfway through a flat interface settles where the
interface meets it at the prescribed angle; its height gives the measured
angle, cos(theta_mes) = (z_i - z_c) / R_p with z_i the far-field interface
height (contact angle measured in phase a, which lies below).

Particle migration in a tube (Sec. V B, the Segre-Silberberg benchmark, in
the body-force-driven periodic form of the 64 x 64 x 1024 configuration): a
neutrally buoyant sphere released off-axis in Poiseuille flow drifts
sideways; the lateral (radial) momentum-exchange force and the radial
position l / R_t are sampled over time.

Detachment set-up (the paper gives R_p = 25, v_p = 0.01 and theta_p from 30 to 150 deg;
the rest is this module's choice): a periodic box of 6 R_p x 6 R_p x 12 R_p
(rounded up to multiples of 8), no substrate, a layer of phase a (the
liquid, phi = +1) between z = R_p / 2 and the flat interface z_i = 4 R_p,
phase b above, equal viscosities 1/6.  The sphere is kinematic: it is held
at the flat-interface equilibrium height z_c = z_i - R_p cos(theta_p) (the
contact angle is measured in phase a) for the equilibration steps, then moved
upwards at v_p until its centre has risen 5 R_p (hydrophilic spheres drag a
liquid bridge that ruptures late).  Only the capillary force
F_sigma of the sphere's record is used.
"""
from __future__ import annotations

import math

import numpy as np

from paper_2505_10171_gb300 import lbm
from paper_2505_10171_gb300 import workloads as W


def _ceil8(v):
    return int(math.ceil(v / 8.0) * 8)


def detachment_setup(theta_deg, R_p):
    """Parameters, order parameter and particle of the detachment benchmark."""
    nx = ny = _ceil8(6 * R_p)
    nz = _ceil8(12 * R_p)
    z_lo, z_i = 0.5 * R_p, 4.0 * R_p
    params = dict(W.COMMON, nx=nx, ny=ny, nz=nz, wall_z0=0, nu_a=1.0 / 6.0, nu_b=1.0 / 6.0)
    z = np.arange(nz, dtype=np.float64)
    d = np.minimum(z - z_lo, z_i - z)  # signed distance into the liquid layer
    prof = np.tanh(2.0 * d / W.INTERFACE_WIDTH)
    phi = np.broadcast_to(prof[:, None, None], (nz, ny, nx)).reshape(-1).copy()
    zc = z_i - R_p * math.cos(math.radians(theta_deg))
    particle = dict(x=(nx / 2.0, ny / 2.0, zc), R=float(R_p), rho_p=W.PARTICLE_DENSITY, theta_deg=float(theta_deg),
                    kinematic=1)
    return params, phi, particle


def detachment(theta_deg, R_p=25, v_p=0.01, equil_steps=None, rise=5.0, sample_every=10, precision="fp32",
               stream=None):
    """Run the benchmark; returns a dict with the sampled times (in units of
    R_p / v_p from the start of the pull), the vertical capillary force, the
    measured maximum F_max = -min F_z, Scheludko's prediction and their ratio.
    The capillary prefactor is the context's default (3 k beta); a prefactor
    C scales F_sigma linearly (the printed (9/2) k beta gives 1.5 times these
    forces)."""
    params, phi, particle = detachment_setup(theta_deg, R_p)
    if equil_steps is None:
        equil_steps = max(400, int(2000 * (R_p / 25.0) ** 2))
    ctx = lbm.Context(params, precision, stream=stream)
    try:
        ctx.lbm_add_particles([particle])
        ctx.lbm_init_fields(phi)
        ctx.lbm_step(equil_steps)
        ctx.lbm_set_particle_motion(0, (0.0, 0.0, v_p))
        n_pull = int(round(rise * R_p / v_p))
        t, fz = [], []
        done = 0
        while done < n_pull:
            k = min(sample_every, n_pull - done)
            ctx.lbm_step(k)
            done += k
            rec = ctx.lbm_particle_forces()[0]
            t.append(done * v_p / R_p)
            fz.append(rec[8])
    finally:
        ctx.close()
    fz = np.asarray(fz)
    f_max = float(-fz.min())
    pred = 2.0 * math.pi * params["sigma"] * R_p * math.cos(math.radians(theta_deg) / 2.0) ** 2
    return dict(theta_deg=theta_deg, R_p=R_p, t=np.asarray(t), Fz=fz, F_max=f_max, F_pred=pred, ratio=f_max / pred,
                t_at_max=float(np.asarray(t)[int(fz.argmin())]), equil_steps=equil_steps)


def interface_height(phi_col):
    """Height of the upper zero crossing of phi along one z column (linear
    interpolation between the two nodes around it: exact for a crossing at a
    node or midway, within 0.03 lattice units for a tanh of width 2.5)."""
    ph = np.asarray(phi_col)
    k = int(np.argmax(ph))
    while k + 1 < len(ph) and ph[k + 1] > 0.0:
        k += 1
    a, b = ph[k], ph[k + 1]
    return k + a / (a - b)


def wetting_equilibrium(theta_deg, R_p=25, steps=None, sample_every=100, precision="fp32", stream=None):
    """Release a free sphere (no gravity) with its centre on a flat interface
    and let it settle.  The box is 8 R_p on each side (the paper's 200^3 at
    R_p = 25), the liquid layer from z = R_p / 2 to z_i = 4 R_p.  Returns the
    sampled times, centre heights and far-field interface heights, and the
    angle measured from the last sample."""
    n = _ceil8(8 * R_p)
    z_lo, z_i = 0.5 * R_p, 4.0 * R_p
    params = dict(W.COMMON, nx=n, ny=n, nz=n, wall_z0=0, nu_a=1.0 / 6.0, nu_b=1.0 / 6.0)
    z = np.arange(n, dtype=np.float64)
    prof = np.tanh(2.0 * np.minimum(z - z_lo, z_i - z) / W.INTERFACE_WIDTH)
    phi = np.broadcast_to(prof[:, None, None], (n, n, n)).reshape(-1).copy()
    particle = dict(x=(n / 2.0, n / 2.0, z_i), R=float(R_p), rho_p=W.PARTICLE_DENSITY, theta_deg=float(theta_deg))
    if steps is None:
        steps = int(16000 * (R_p / 25.0) ** 2)
    ctx = lbm.Context(params, precision, stream=stream)
    try:
        ctx.lbm_add_particles([particle])
        ctx.lbm_init_fields(phi)
        t, zc, zi = [], [], []
        done = 0
        while done < steps:
            k = min(sample_every, steps - done)
            ctx.lbm_step(k)
            done += k
            t.append(done)
            zc.append(ctx.lbm_particle_forces()[0][20])
        f = ctx.lbm_read_fields(lbm.FIELD_PHI).reshape(n, n, n)
        zi_far = float(np.mean([interface_height(f[:, y, x]) for y, x in ((0, 0), (0, n // 2), (n // 2, 0))]))
    finally:
        ctx.close()
    zc = np.asarray(zc)
    c = (zi_far - zc[-1]) / R_p
    theta_mes = math.degrees(math.acos(max(-1.0, min(1.0, c))))
    return dict(theta_deg=theta_deg, R_p=R_p, t=np.asarray(t), z_c=zc, z_i=zi_far, theta_mes=theta_mes)


def tube_migration(nz=1024, steps=50000, sample_every=500, precision="fp32", stream=None):
    """The tube workload (radius 31 about (31.5, 31.5), periodic along z, body
    force for a centreline speed of 0.02, sphere R_p = 6 released at
    l = 0.3 R_t with the local flow speed).  Returns the sampled times, the
    radial position l / R_t, the radial and axial momentum-exchange forces and
    the axial flow speed on the tube axis far from the sphere at the end."""
    w = W.cfg3(nz=nz)
    Rt, c0 = 31.0, 31.5
    ctx = lbm.Context(dict(w["params"], store_velocity=1), precision, stream=stream)
    try:
        ctx.lbm_set_solid_mask(w["mask"])
        ctx.lbm_add_particles(w["particles"])
        ctx.lbm_init_fields(w["phi"], None, w["u"])
        t, l, fr, fz = [], [], [], []
        done = 0
        while done < steps:
            k = min(sample_every, steps - done)
            ctx.lbm_step(k)
            done += k
            rec = ctx.lbm_particle_forces()[0]
            d = np.array([rec[18] - c0, rec[19] - c0])
            r = float(np.hypot(*d))
            e = d / max(r, 1e-12)
            t.append(done)
            l.append(r / Rt)
            fr.append(float(rec[0] * e[0] + rec[1] * e[1]))
            fz.append(float(rec[2]))
        zp = rec[20]
        u = ctx.lbm_read_fields(lbm.FIELD_U).reshape(3, nz, 64, 64)
        zf = int((zp + nz / 2) % nz)  # the plane farthest from the sphere
        u_axis = float(u[2, zf, 31:33, 31:33].mean())
    finally:
        ctx.close()
    return dict(t=np.asarray(t), l=np.asarray(l), F_r=np.asarray(fr), F_z=np.asarray(fz), u_axis=u_axis)


def tube_pressure_migration(steps=100000, sample_every=1000, nz=2560, precision="fp32", stream=None, **kw):
    """The Segre-Silberberg benchmark of Sec. V D at the paper's parameters
    (R_t = 40, R_p = 12.2, rho_f = 1.05, nu = 0.457, mean inlet speed 0.0113,
    release at l = 0.21 R_t), driven by anti-bounce-back pressure faces at
    both ends of a tube nz long.  Returns the sampled times, l / R_t, the
    sphere's axial position, and the mean axial speed over a cross-section far
    from the sphere at the end (against the imposed 0.0113); stops early when
    the sphere comes within 2 R_p of the outlet face."""
    w = W.tube_pressure(nz=nz, **kw)
    c, Rt, Rp = w["centre"], w["R_t"], w["particles"][0]["R"]
    ny = nx = w["params"]["nx"]
    ctx = lbm.Context(dict(w["params"], store_velocity=1), precision, stream=stream)
    try:
        ctx.lbm_set_solid_mask(w["mask"])
        ctx.lbm_add_particles(w["particles"])
        ctx.lbm_init_fields(w["phi"], w["rho"], w["u"])
        t, l, zs = [], [], []
        done = 0
        while done < steps:
            k = min(sample_every, steps - done)
            ctx.lbm_step(k)
            done += k
            rec = ctx.lbm_particle_forces()[0]
            t.append(done)
            l.append(float(np.hypot(rec[18] - c, rec[19] - c)) / Rt)
            zs.append(float(rec[20]))
            if rec[20] > nz - 1.5 - 2 * Rp:
                break
        u = ctx.lbm_read_fields(lbm.FIELD_U).reshape(3, nz, ny, nx)
        own = ctx.owner().reshape(nz, ny, nx)
        zf = int(zs[-1] - nz / 2) % (nz - 4) + 2 if zs[-1] > nz / 2 else int(zs[-1] + nz / 2)
        zf = min(max(zf, 2), nz - 3)
        sec = own[zf] == 0
        u_mean = float(u[2, zf][sec].mean())
    finally:
        ctx.close()
    return dict(t=np.asarray(t), l=np.asarray(l), z=np.asarray(zs), u_mean=u_mean, v_in=kw.get("v_in", 0.0113))


# outcomes of a drop-particle collision (Sec. VI B/C)
PUSH_PULL, ENTER_EXIT, CAPTURED_AFTER_ENTERING, NO_CONTACT, LEFT_BEHIND = (
    "push-pull", "enter-exit", "captured after entering", "no contact", "left behind")


def classify_outcome(shell_phi, inside=0.5):
    """Outcome of one collision from the order parameter sampled on the
    sphere's shell (rows: samples in time, columns: shell points; phase a,
    phi > 0, is the drop).  The particle touches the drop when some shell
    point is in phase a, is inside it when the shell's mean phi exceeds
    `inside`.  Captured (the particle stays attached to the drop) = touching
    at the last sample.  push-pull: captured, never inside; enter-exit:
    inside at some sample, detached at the end; captured after entering;
    left behind: touched, never inside, detached; no contact: never touched."""
    s = np.asarray(shell_phi, dtype=float)
    touch = (s > 0.0).any(axis=1)
    entered = bool((s.mean(axis=1) > inside).any())
    captured = bool(touch[-1])
    if not touch.any():
        return NO_CONTACT
    if captured:
        return CAPTURED_AFTER_ENTERING if entered else PUSH_PULL
    return ENTER_EXIT if entered else LEFT_BEHIND


def capture_map(mus, mu_rs, steps=40000, sample_every=500, precision="fp16", stream=None, **kw):
    """The friction map of Sec. VI C on the batched sweep: one instance per
    (mu, mu_r) of workloads.capture_case, all stepped in one context (one
    launch per kernel per step, graph-captured); every sample_every steps the
    shell order parameter of each sphere (the surrogate's shell features) and
    its record are read.  Returns per case mu, mu_r, the outcome, the sphere's
    x displacement and its rolling ratio omega_y R_p / v_x at the end."""
    cases = [(m, r) for m in mus for r in mu_rs]
    ws = [W.capture_case(m, r, **kw) for m, r in cases]
    # the shell features read the stored collision velocity
    ctx = lbm.Context([dict(w["params"], store_velocity=1) for w in ws], precision, stream=stream)
    try:
        for k, w in enumerate(ws):
            ctx.lbm_add_particles(w["particles"], inst=k)
            ctx.lbm_init_fields(w["phi"], inst=k)
        x0 = [ctx.lbm_particle_forces(k)[0][18] for k in range(len(ws))]
        shells = [[] for _ in ws]
        done = 0
        while done < steps:
            n = min(sample_every, steps - done)
            ctx.lbm_step(n)
            done += n
            for k in range(len(ws)):
                f = ctx.lbm_surrogate_features(k)[0]
                shells[k].append(f[0:4 * 96:4])  # phi at the 96 shell points
        out = []
        for k, (m, r) in enumerate(cases):
            rec = ctx.lbm_particle_forces(k)[0]
            nx = ws[k]["params"]["nx"]
            dx = (rec[18] - x0[k] + nx / 2) % nx - nx / 2
            v, wv = rec[21:24], rec[24:27]
            out.append(dict(mu=m, mu_r=r, outcome=classify_outcome(shells[k]), dx=float(dx),
                            rolling=float(wv[1] * ws[k]["particles"][0]["R"] / v[0]) if abs(v[0]) > 1e-9 else 0.0))
    finally:
        ctx.close()
    return out


def main():
    """Command line: run one of the long set-ups and write its record (JSON)."""
    import argparse
    import json
    import sys
    import time
    ap = argparse.ArgumentParser(description="long validation runs of the method, through the C ABI")
    sub = ap.add_subparsers(dest="case", required=True)
    t = sub.add_parser("tube-pressure", help="Segre-Silberberg tube with pressure faces (Sec. V B, V D)")
    t.add_argument("--steps", type=int, default=116000)
    t.add_argument("--every", type=int, default=2000)
    m = sub.add_parser("friction-map", help="collision outcomes over (mu, mu_r) (Sec. VI C)")
    m.add_argument("--steps", type=int, default=40000)
    m.add_argument("--every", type=int, default=1000)
    m.add_argument("--grid", default="0,0.2,0.4,0.6,0.8,1.0", help="values of mu and of mu_r")
    ap.add_argument("--out", required=True, help="JSON record to write")
    a = ap.parse_args()
    t0 = time.time()
    if a.case == "tube-pressure":
        r = tube_pressure_migration(steps=a.steps, sample_every=a.every)
        rec = dict(t=[int(v) for v in r["t"]], l_over_Rt=[round(float(v), 5) for v in r["l"]],
                   axial_position=[round(float(v), 2) for v in r["z"]], u_mean_far=r["u_mean"], v_in=r["v_in"])
    else:
        grid = [float(v) for v in a.grid.split(",")]
        rec = dict(cases=capture_map(grid, grid, steps=a.steps, sample_every=a.every))
    rec["seconds"] = time.time() - t0
    rec["command"] = "python -m paper_2505_10171_gb300.validation " + " ".join(sys.argv[1:])
    json.dump(rec, open(a.out, "w"), indent=1)
    print(json.dumps(rec)[:2000])


if __name__ == "__main__":
    main()
