"""Training and evaluation campaign of the learned force surrogate on coarse
grids, through the C ABI.

Resolved runs of a 256 x 128 x 128 drop-sphere set-up (R_p = 8, see
_setup) give the labels: every `every` steps, each sphere's resolved fluid
force and torque (momentum exchange plus capillary), divided by sigma R_p and
sigma R_p^2.  The coarse set-ups are the same runs at 3/8 scale (96 x 48 x 48,
drop R = 15, R_p = 3, U and sigma scaled by 3/8, viscosities kept: diffusive
scaling, so that t U / R_p and the step count match).  Held-out seeds run on
the coarse grid with the plain coarse forces and with the surrogate, and both
are compared with the resolved runs of the same seeds at the same steps.

Choices (the paper has no surrogate): the shell has radius 1.5 R_p on either
grid; velocities are scaled by each run's drop speed target U and radii by
R_p.  The network's inputs come from one of two sources:
  inputs="coarse" (default): the shells of the coarse run of the same seed at
    the same step, paired with the resolved labels, so that training and use
    see the same grid;
  inputs="box": the resolved run's own shells, box-filtered over one coarse
    cell (width 8/3 resolved units, 27-point midpoint rule), the reading that
    restricts resolved fields to the coarse resolution.  Measured at 8
    training and 8 held-out seeds, the network fitted this way is accurate on
    resolved inputs but worse than the plain coarse method on coarse ones: the
    coarse grid's interface is 8/3 times wider in physical units and its
    near-sphere flow differs, which a box filter of the resolved fields does
    not reproduce.
The spheres are held at rest on the substrate (prescribed motion) while the
drop sweeps over them, so that the resolved and coarse runs of a seed have
the same particle positions at every sample: the comparison measures the
force model alone, and the pairing of inputs and labels is exact in geometry.

Acoustics: the start-up sends pressure waves through the weakly damped
ambient phase, which load every sphere by up to 0.2 sigma R_p long before
the drop arrives.  Their periods are set by the box size over the lattice
sound speed, so they do not follow the diffusive scaling between the grids
and the two grids' waves are out of phase at matched steps (measured: on
the 92% of samples where no sphere touches the drop, the resolved and
coarse forces are uncorrelated).  Labels and every compared force series are
therefore also taken through a centred moving average over `smooth` samples
(default 64 samples of 16 steps, above the 256-unit box's longest acoustic
period of about 890 steps), and the errors are reported raw and smoothed,
over all samples and over the samples where the sphere touches the drop.
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import numpy as np

from paper_2505_10171_gb300 import lbm
from paper_2505_10171_gb300 import workloads as W

SCALE = 3.0 / 8.0
FINE_U, FINE_RP = 5.0e-3, 8.0
SHELL = 0.5            # shell radius (1 + SHELL) R_p
BOX = 1.0 / SCALE      # box filter of the resolved inputs: one coarse cell
# nodes per context: 38 N must stay below 2^31 (population indices are int32)
MAX_NODES = 50_000_000


def _setup(seed, s, free=False, box=0.0, moving=False):
    """Drop R = 40 s driven along x at 5e-3 s over a 150 deg wall, eight
    spheres R_p = 8 s (contact angles uniform in [30, 90] deg) placed 4 to 50 s
    ahead of the drop front (centres x in [98, 152] s, y in [12, 116] s) at
    centre spacings of at least 24 s, on a box of 256 x 128 x 128 times s.
    The contact offset delta_R stays one lattice unit.  Held spheres
    (free=False) sit at rest one delta_R above the wall.  Free spheres rest
    on the wall with normal damping at half the critical value and a weight
    of 2 sigma R_p: a sphere must keep a fluid node between itself and the
    wall, or the momentum exchange on its open surface carries the
    unbalanced rest pressure.  Moving (held spheres only): all spheres of the
    seed glide along the substrate with one prescribed velocity, x component
    uniform in [-U, U], y component uniform in [-U/3, U/3] (U the drop speed
    target), rolling without slip on odd seeds, so that the network also sees
    spheres that move relative to the fluid."""
    rng = np.random.default_rng(seed)
    R8, Rc8 = FINE_RP, FINE_RP + 1.0
    centres = W.place_spheres(rng, 8, R8, Rc8, (98.0, 152.0), (12.0, 116.0), 9.5, 24.0)
    thetas = rng.uniform(30.0, 90.0, size=8)
    glide = np.array([rng.uniform(-1.0, 1.0), rng.uniform(-1.0 / 3.0, 1.0 / 3.0), 0.0]) * FINE_U * s
    nx, ny, nz = int(round(256 * s)), int(round(128 * s)), int(round(128 * s))
    sigma, R_p = W.COMMON["sigma"] * s, R8 * s
    gn = W.resting_damping(R_p)
    params = dict(W.COMMON, nx=nx, ny=ny, nz=nz, wall_z0=1, theta_wall_deg=150.0, nu_a=1.0 / 6.0,
                  nu_b=1.0 / 60.0, mu_s=0.3, mu_r=0.05, gn=gn, sigma=sigma, delta_R=1.0,
                  body_force_a=(2.0e-6 * s, 0.0, 0.0), g_particle=(0.0, 0.0, -2.0 * sigma * R_p),
                  drop_speed_control=1, drop_speed_target=(FINE_U * s, 0.0, 0.0), drop_speed_interval=100,
                  store_velocity=1, surrogate_u_ref=FINE_U * s, surrogate_r_ref=R_p,
                  surrogate_shell_gap=SHELL * R_p, surrogate_box=box)
    phi = W.drop_phi(nx, ny, nz, (48.0 * s, 64.0 * s, 0.5), 40.0 * s)
    particles = [dict(x=(c[0] * s, c[1] * s, 0.5 + R_p + 1.0), R=R_p, rho_p=W.PARTICLE_DENSITY,
                      theta_deg=float(t), kinematic=0 if free else 1) for c, t in zip(centres, thetas)]
    if moving and not free:
        roll = seed % 2 == 1
        w = (-glide[1] / R_p, glide[0] / R_p, 0.0) if roll else (0.0, 0.0, 0.0)
        for q in particles:
            q["v"] = tuple(float(v) for v in glide)
            q["w"] = tuple(float(v) for v in w)
    return dict(params=params, phi=phi, particles=particles)


def resolved(seed, free=False, box=BOX, moving=False):
    """The resolved (R_p = 8) set-up of a seed (shell inputs box-filtered)."""
    return _setup(seed, 1.0, free, box, moving)


def coarse(seed, free=False, moving=False):
    """The same set-up at 3/8 scale (R_p = 3)."""
    return _setup(seed, SCALE, free, moving=moving)


def _labels(rec, sigma, R_p):
    F = rec[:, 0:3] + rec[:, 6:9]
    T = rec[:, 3:6] + rec[:, 9:12]
    return np.concatenate([F / (sigma * R_p), T / (sigma * R_p * R_p)], axis=1)


def _chunks(ws):
    """Split the workloads into contexts of at most MAX_NODES nodes, as even
    in count as the limit allows."""
    nodes = [w["params"]["nx"] * w["params"]["ny"] * w["params"]["nz"] for w in ws]
    per = max(1, int(MAX_NODES // max(nodes)))
    n = math.ceil(len(ws) / per)
    base, extra = divmod(len(ws), n)
    out, i = [], 0
    for k in range(n):
        size = base + (1 if k < extra else 0)
        out.append(list(range(i, i + size)))
        i += size
    return out


def run(ws, steps, every, weights=None, features=True, stream=None):
    """Step the workloads ws (batched, one instance each, in as few contexts
    as the node limit allows) and sample every `every` steps.  Returns per
    instance the inputs X [samples][387] (when features) and the
    nondimensional fluid force and torque Y [samples][6], samples ordered by
    time then sphere.  With weights, the contexts use the surrogate for the
    particle forces."""
    out = [None] * len(ws)
    for idx in _chunks(ws):
        part = [ws[i] for i in idx]
        ctx = lbm.Context([w["params"] for w in part], "fp32", stream=stream)
        try:
            for k, w in enumerate(part):
                ctx.lbm_add_particles(w["particles"], inst=k)
                ctx.lbm_init_fields(w["phi"], inst=k)
            if weights is not None:
                ctx.lbm_surrogate_load(weights)
                ctx.lbm_set_force_model(lbm.FORCE_SURROGATE)
            X = [[] for _ in part]
            Y = [[] for _ in part]
            done = 0
            while done < steps:
                ctx.lbm_step(every)
                done += every
                for k, w in enumerate(part):
                    if features:
                        X[k].append(ctx.lbm_surrogate_features(k))
                    Y[k].append(_labels(ctx.lbm_particle_forces(k), w["params"]["sigma"], w["particles"][0]["R"]))
        finally:
            ctx.close()
        for k, i in enumerate(idx):
            out[i] = dict(X=np.concatenate(X[k]) if features else None, Y=np.concatenate(Y[k]))
    return out


def errors(Y, Yref, mask=None):
    """Mean over samples (those of mask, when given) of |F - F_ref| and
    |T - T_ref| (nondimensional)."""
    m = np.ones(len(Y), bool) if mask is None else mask
    if not m.any():
        return (float("nan"), float("nan"))
    return (float(np.linalg.norm(Y[m, 0:3] - Yref[m, 0:3], axis=1).mean()),
            float(np.linalg.norm(Y[m, 3:6] - Yref[m, 3:6], axis=1).mean()))


def smooth(Y, n_sph, win):
    """Centred moving average over `win` samples of each sphere's series
    (Y: [samples][k], time-major with n_sph spheres per time), the window
    shortened at the ends; same shape as Y."""
    if win <= 1:
        return Y
    T = len(Y) // n_sph
    A = Y.reshape(T, n_sph, -1)
    c = np.concatenate([np.zeros((1,) + A.shape[1:]), np.cumsum(A, axis=0)])
    h = win // 2
    lo = np.clip(np.arange(T) - h, 0, T)
    hi = np.clip(np.arange(T) - h + win, 0, T)
    return ((c[hi] - c[lo]) / (hi - lo)[:, None, None]).reshape(Y.shape)


def touching(X):
    """Samples whose shell reaches the drop (some shell point with phi > 0)."""
    return (X[:, 0:384:4] > 0.0).any(axis=1)


def init_weights(seed):
    """Uniform +-1/sqrt(fan-in) weights, zero biases and padding columns."""
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
    return th


def campaign(train_seeds, test_seeds, steps=16000, every=16, epochs=40, batch=512, lr=1e-3, seed=9, free=False,
             inputs="coarse", win=64, moving=False, stream=None):
    """Train on train_seeds (labels: their resolved runs' forces through the
    moving average over `win` samples; inputs as `inputs` says), then compare
    on test_seeds: the network offline on the test inputs, and the coarse runs
    with the plain forces and with the surrogate in the loop, all against the
    resolved test runs, raw and smoothed, on all samples and on those where
    the sphere touches the drop in the coarse run.  The learning rate halves
    after half and after three quarters of the epochs.  Returns the error
    table and the training record (losses, weights)."""
    if inputs not in ("coarse", "box"):
        raise ValueError("inputs must be 'coarse' or 'box'")
    box = inputs == "box"
    n_sph = 8
    t0 = time.time()
    tr = run([resolved(sd, free, moving=moving) for sd in train_seeds], steps, every, features=box, stream=stream)
    Y = np.concatenate([smooth(r["Y"], n_sph, win) for r in tr])
    if box:
        X = np.concatenate([r["X"] for r in tr])
    else:
        trc = run([coarse(sd, free, moving=moving) for sd in train_seeds], steps, every, stream=stream)
        X = np.concatenate([r["X"] for r in trc])
        del trc
    del tr
    t_train_data = time.time() - t0
    ref = run([resolved(sd, free) for sd in test_seeds], steps, every, features=box, stream=stream)
    t_ref = time.time() - t0 - t_train_data
    cws = [coarse(sd, free) for sd in test_seeds]
    t2 = time.time()
    plain = run(cws, steps, every, stream=stream)
    t_plain = time.time() - t2
    test_X = [r["X"] for r in (ref if box else plain)]
    # the network lives in a context; a small coarse one hosts it
    host = lbm.Context(cws[0]["params"], "fp32", stream=stream)
    try:
        host.lbm_surrogate_load(init_weights(seed))
        losses = []
        t1 = time.time()
        for e in range(epochs):
            rate = lr * (0.5 if e >= epochs // 2 else 1.0) * (0.5 if e >= (3 * epochs) // 4 else 1.0)
            losses.append(host.lbm_surrogate_train(X, Y, 1, batch, rate, seed + e))
        t_fit = time.time() - t1
        weights = host.lbm_surrogate_save()
        pred = [np.concatenate([host.lbm_surrogate_predict(x[i:i + lbm.MLP_MAX_BATCH])
                                for i in range(0, len(x), lbm.MLP_MAX_BATCH)]).astype(np.float64)
                for x in test_X]
    finally:
        host.close()
    t3 = time.time()
    sur = run(cws, steps, every, weights=weights, features=False, stream=stream)
    t_sur = time.time() - t3
    series = dict(offline=pred, plain_coarse=[p["Y"] for p in plain], surrogate_coarse=[p["Y"] for p in sur])
    touch = np.concatenate([touching(p["X"]) for p in plain])
    table = dict(inputs=inputs, moving_training=bool(moving), samples=int(X.shape[0]), test_samples=int(len(touch)),
                 touching_fraction=float(touch.mean()), train_seeds=len(train_seeds), test_seeds=len(test_seeds),
                 steps=steps, every=every, smooth_window=win, epochs=epochs, free=bool(free),
                 label_rms=float(np.sqrt((Y * Y).mean())), loss_first=losses[0], loss_last=losses[-1])
    for tag, w_ in (("raw", 1), ("smoothed", win)):
        Yr = np.concatenate([smooth(r["Y"], n_sph, w_) for r in ref])
        table[f"ref_force_mean_{tag}"] = float(np.linalg.norm(Yr[:, 0:3], axis=1).mean())
        table[f"ref_force_mean_touching_{tag}"] = (float(np.linalg.norm(Yr[touch, 0:3], axis=1).mean()) if touch.any() else float("nan"))
        for name, rows in series.items():
            Ys = np.concatenate([smooth(y, n_sph, w_) for y in rows])
            table[f"{name}_{tag}"] = list(errors(Ys, Yr))
            table[f"{name}_touching_{tag}"] = list(errors(Ys, Yr, touch))
    table["seconds"] = dict(train_data=t_train_data, reference=t_ref, fit=t_fit, plain_coarse=t_plain,
                            surrogate_coarse=t_sur)
    return table, dict(losses=losses, weights=weights)


def evaluate(weights, test_seeds, steps=16000, every=16, free=False, win=64, stream=None):
    """Run trained weights on test_seeds without training: the resolved
    runs, and the coarse runs with the plain forces and with the surrogate in
    the loop; the error table as campaign() reports it (no offline column)."""
    n_sph = 8
    t0 = time.time()
    ref = run([resolved(sd, free) for sd in test_seeds], steps, every, features=False, stream=stream)
    cws = [coarse(sd, free) for sd in test_seeds]
    plain = run(cws, steps, every, stream=stream)
    sur = run(cws, steps, every, weights=weights, features=False, stream=stream)
    series = dict(plain_coarse=[p["Y"] for p in plain], surrogate_coarse=[p["Y"] for p in sur])
    touch = np.concatenate([touching(p["X"]) for p in plain])
    table = dict(test_samples=int(len(touch)), touching_fraction=float(touch.mean()), test_seeds=len(test_seeds),
                 steps=steps, every=every, smooth_window=win, free=bool(free))
    for tag, w_ in (("raw", 1), ("smoothed", win)):
        Yr = np.concatenate([smooth(r["Y"], n_sph, w_) for r in ref])
        table[f"ref_force_mean_{tag}"] = float(np.linalg.norm(Yr[:, 0:3], axis=1).mean())
        table[f"ref_force_mean_touching_{tag}"] = (float(np.linalg.norm(Yr[touch, 0:3], axis=1).mean()) if touch.any() else float("nan"))
        for name, rows in series.items():
            Ys = np.concatenate([smooth(y, n_sph, w_) for y in rows])
            table[f"{name}_{tag}"] = list(errors(Ys, Yr))
            table[f"{name}_touching_{tag}"] = list(errors(Ys, Yr, touch))
    table["seconds"] = time.time() - t0
    return table


def main():
    ap = argparse.ArgumentParser(description="surrogate training and coarse-grid evaluation campaign")
    ap.add_argument("--train", type=int, default=25, help="resolved training runs (seeds 1..N)")
    ap.add_argument("--test", type=int, default=64, help="held-out seeds (1001..) run coarse and resolved")
    ap.add_argument("--steps", type=int, default=16000)
    ap.add_argument("--every", type=int, default=16)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--free", action="store_true", help="free spheres instead of held ones")
    ap.add_argument("--inputs", choices=("coarse", "box"), default="coarse",
                    help="network inputs: coarse-run shells, or box-filtered resolved shells")
    ap.add_argument("--smooth", type=int, default=64, help="moving-average window in samples")
    ap.add_argument("--moving", action="store_true", help="train on spheres gliding on prescribed paths")
    ap.add_argument("--out", default=None, help="write the error table as JSON here")
    ap.add_argument("--weights", default=None, help="write the trained FP32 weights (.npy) here")
    ap.add_argument("--evaluate", default=None, help="evaluate these weights (.npy) instead of training")
    a = ap.parse_args()
    if a.evaluate:
        table = evaluate(np.load(a.evaluate), list(range(1001, 1001 + a.test)), steps=a.steps, every=a.every,
                         free=a.free, win=a.smooth)
        table["weights"] = a.evaluate
        table["command"] = "python -m paper_2505_10171_gb300.surrogate_study " + " ".join(sys.argv[1:])
        print(json.dumps(table))
        if a.out:
            json.dump(table, open(a.out, "w"), indent=1)
        return
    table, rec = campaign(list(range(1, a.train + 1)), list(range(1001, 1001 + a.test)), steps=a.steps,
                          every=a.every, epochs=a.epochs, free=a.free, inputs=a.inputs, win=a.smooth,
                          moving=a.moving)
    table["losses"] = rec["losses"]
    table["command"] = "python -m paper_2505_10171_gb300.surrogate_study " + " ".join(sys.argv[1:])
    print(json.dumps(table))
    if a.out:
        json.dump(table, open(a.out, "w"), indent=1)
    if a.weights:
        np.save(a.weights, rec["weights"])


if __name__ == "__main__":
    main()
