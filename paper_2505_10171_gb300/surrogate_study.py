"""Training and evaluation campaign of the learned force surrogate on coarse
grids, through the C ABI.

Resolved runs of a 256 x 128 x 128 drop-sphere set-up (R_p = 8, see
_setup) give the training samples: every `every` steps, the 387 shell inputs
of each sphere and its resolved fluid force and torque (momentum exchange
plus capillary), divided by sigma R_p and sigma R_p^2.  The test set-ups are
the same runs at 3/8 scale (96 x 48 x 48, drop R = 15, R_p = 3, U and sigma
scaled by 3/8, viscosities kept: diffusive scaling, so that t U / R_p and
the step count match).  They run twice on the coarse grid, with the plain coarse
forces and with the surrogate, and both are compared with the resolved runs
of the same seeds at the same steps.

Choices (the paper has no surrogate): the shell lies at R_p + 2 coarse units,
the resolved samples use the same physical shell (R_p + 16/3 fine units);
velocities are scaled by each run's drop speed target U and radii by R_p; the
resolved inputs are taken on the resolved run's own fields by the GPU feature
kernel (no box filter).
"""
from __future__ import annotations

import numpy as np

from paper_2505_10171_gb300 import lbm
from paper_2505_10171_gb300 import workloads as W

SCALE = 3.0 / 8.0
FINE_U, FINE_RP, SHELL_GAP = 5.0e-3, 8.0, 2.0


def _setup(seed, s):
    """Drop R = 40 s driven along x at 5e-3 s over a 150 deg wall, eight
    spheres R_p = 8 s (contact angles uniform in [30, 90] deg) placed 4 to 50 s
    ahead of the drop front (centres x in [98, 152] s, y in [12, 116] s) at
    centre spacings of at least 24 s, on a box of
    256 x 128 x 128 times s.  The contact offset delta_R stays one lattice unit
    and the spheres rest on the wall with normal damping at half the critical
    value and a weight of 2 sigma R_p: a sphere must keep a fluid node
    between itself and the wall, or the momentum exchange on its open surface
    carries the unbalanced rest pressure (with the weight 10 sigma R_p and no
    damping of the 256 x 128 x 128 benchmark workload, spheres that overshoot
    their rest overlap seal against the wall and are pushed into it)."""
    rng = np.random.default_rng(seed)
    R8, Rc8 = FINE_RP, FINE_RP + 1.0
    centres = W.place_spheres(rng, 8, R8, Rc8, (98.0, 152.0), (12.0, 116.0), 9.5, 24.0)
    thetas = rng.uniform(30.0, 90.0, size=8)
    nx, ny, nz = int(round(256 * s)), int(round(128 * s)), int(round(128 * s))
    sigma, R_p = W.COMMON["sigma"] * s, R8 * s
    gn = W.resting_damping(R_p)
    params = dict(W.COMMON, nx=nx, ny=ny, nz=nz, wall_z0=1, theta_wall_deg=150.0, nu_a=1.0 / 6.0,
                  nu_b=1.0 / 60.0, mu_s=0.3, mu_r=0.05, gn=gn, sigma=sigma, delta_R=1.0,
                  body_force_a=(2.0e-6 * s, 0.0, 0.0), g_particle=(0.0, 0.0, -2.0 * sigma * R_p),
                  drop_speed_control=1, drop_speed_target=(FINE_U * s, 0.0, 0.0), drop_speed_interval=100,
                  store_velocity=1, surrogate_u_ref=FINE_U * s, surrogate_r_ref=R_p,
                  surrogate_shell_gap=SHELL_GAP * (s / SCALE))
    phi = W.drop_phi(nx, ny, nz, (48.0 * s, 64.0 * s, 0.5), 40.0 * s)
    particles = [dict(x=(c[0] * s, c[1] * s, 0.5 + R_p + 1.0), R=R_p, rho_p=W.PARTICLE_DENSITY,
                      theta_deg=float(t)) for c, t in zip(centres, thetas)]
    return dict(params=params, phi=phi, particles=particles)


def resolved(seed):
    """The resolved (R_p = 8) set-up of a seed."""
    return _setup(seed, 1.0)


def coarse(seed):
    """The same set-up at 3/8 scale (R_p = 3)."""
    return _setup(seed, SCALE)


def _labels(rec, sigma, R_p):
    F = rec[:, 0:3] + rec[:, 6:9]
    T = rec[:, 3:6] + rec[:, 9:12]
    return np.concatenate([F / (sigma * R_p), T / (sigma * R_p * R_p)], axis=1)


def run(ws, steps, every, weights=None, features=True, stream=None):
    """Step the workloads ws (one context, one instance each) and sample every
    `every` steps.  Returns per instance the inputs X [samples][387] (when
    features) and the nondimensional fluid force and torque Y [samples][6],
    samples ordered by time then sphere.  With weights, the context uses the
    surrogate for the particle forces."""
    ctx = lbm.Context([w["params"] for w in ws], "fp32", stream=stream)
    try:
        for k, w in enumerate(ws):
            ctx.lbm_add_particles(w["particles"], inst=k)
            ctx.lbm_init_fields(w["phi"], inst=k)
        if weights is not None:
            ctx.lbm_surrogate_load(weights)
            ctx.lbm_set_force_model(lbm.FORCE_SURROGATE)
        X = [[] for _ in ws]
        Y = [[] for _ in ws]
        done = 0
        while done < steps:
            ctx.lbm_step(every)
            done += every
            for k, w in enumerate(ws):
                p = w["params"]
                R_p = w["particles"][0]["R"]
                if features:
                    X[k].append(ctx.lbm_surrogate_features(k))
                Y[k].append(_labels(ctx.lbm_particle_forces(k), p["sigma"], R_p))
    finally:
        ctx.close()
    out = []
    for k in range(len(ws)):
        out.append(dict(X=np.concatenate(X[k]) if features else None, Y=np.concatenate(Y[k])))
    return out


def errors(Y, Yref):
    """Mean over samples of |F - F_ref| and |T - T_ref| (nondimensional)."""
    return (float(np.linalg.norm(Y[:, 0:3] - Yref[:, 0:3], axis=1).mean()),
            float(np.linalg.norm(Y[:, 3:6] - Yref[:, 3:6], axis=1).mean()))


def campaign(train_seeds, test_seeds, steps=16000, every=32, epochs=40, batch=512, lr=1e-3, seed=9,
             stream=None):
    """Train on the resolved runs of train_seeds, then compare on test_seeds:
    the network on the resolved test inputs (offline), and the coarse runs
    with the plain forces and with the surrogate, all against the resolved
    test runs.  Returns the error table and the training record."""
    Xs, Ys = [], []
    for sd in train_seeds:
        r = run([resolved(sd)], steps, every, stream=stream)[0]
        Xs.append(r["X"])
        Ys.append(r["Y"])
    X, Y = np.concatenate(Xs), np.concatenate(Ys)
    ref = [run([resolved(sd)], steps, every, stream=stream)[0] for sd in test_seeds]
    cws = [coarse(sd) for sd in test_seeds]
    # the network lives in a context; train it in the plain coarse one's place
    host = lbm.Context(cws[0]["params"], "fp32", stream=stream)
    # initial weights: uniform +-1/sqrt(fan-in), zero biases and padding columns
    rng = np.random.default_rng(seed)
    th = np.zeros(lbm.MLP_PARAMS, dtype=np.float32)
    o = 0
    for rows, cols, fan in ((128, 400, 387), (128, 0, 0), (128, 128, 128), (128, 0, 0), (6, 128, 128), (6, 0, 0)):
        n = rows * cols if cols else rows
        if cols:
            a = 1.0 / np.sqrt(fan)
            blk = rng.uniform(-a, a, size=(rows, cols)).astype(np.float32)
            if cols == 400:
                blk[:, 387:] = 0.0
            th[o:o + n] = blk.reshape(-1)
        o += n
    host.lbm_surrogate_load(th)
    losses = [host.lbm_surrogate_train(X, Y, 1, batch, lr, seed + e) for e in range(epochs)]
    weights = host.lbm_surrogate_save()
    off = []
    for r in ref:
        pred = np.concatenate([host.lbm_surrogate_predict(r["X"][i:i + lbm.MLP_MAX_BATCH])
                               for i in range(0, len(r["X"]), lbm.MLP_MAX_BATCH)])
        off.append(errors(pred.astype(np.float64), r["Y"]))
    host.close()
    plain = run(cws, steps, every, features=False, stream=stream)
    sur = run(cws, steps, every, weights=weights, features=False, stream=stream)
    table = dict(samples=int(X.shape[0]), label_rms=float(np.sqrt((Y * Y).mean())),
                 offline=np.mean(off, axis=0).tolist(),
                 plain_coarse=np.mean([errors(plain[k]["Y"], ref[k]["Y"]) for k in range(len(cws))], axis=0).tolist(),
                 surrogate_coarse=np.mean([errors(sur[k]["Y"], ref[k]["Y"]) for k in range(len(cws))],
                                          axis=0).tolist(),
                 ref_force_mean=float(np.mean([np.linalg.norm(r["Y"][:, 0:3], axis=1).mean() for r in ref])))
    return table, dict(losses=losses, weights=weights)
