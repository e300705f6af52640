"""FP64 NumPy reference of the learned particle-force surrogate.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU legs may use this module.  Nothing in the library imports
it and it imports nothing from the library.

The surrogate (an extension of the method, not in the paper) replaces the
momentum-exchange and capillary forces on a coarse grid by a small network
evaluated on samples of the flow around each sphere:

* features (387, zero-padded to 400): on a shell of radius R_p + gap around
  the particle centre, 96 points of a Fibonacci sphere; at each point the
  order parameter and the fluid velocity relative to the particle's rigid-body
  motion, u - (v_p + w_p x (X - x_p)), divided by a reference speed; then
  cos(theta_p), sin(theta_p) and R_p / R_ref.  Fields at a point are
  trilinear interpolations over the fluid corners of its lattice cell (weights
  renormalised; no fluid corner -> zeros), as for the capillary force.
* network: h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = W3 h2 + b3 with
  400 -> 128 -> 128 -> 6; y = (F / (sigma R_p), T / (sigma R_p^2)).
* loss: mean over the samples of a batch and the 6 outputs of the squared
  error.
* optimiser: Adam (Kingma and Ba, 2015): m <- b1 m + (1 - b1) g,
  v <- b2 v + (1 - b2) g^2, p <- p - lr m/(1 - b1^t) / (sqrt(v/(1 - b2^t)) + eps),
  b1 = 0.9, b2 = 0.999, eps = 1e-8.
* batches: each epoch visits the samples in the order of a Fisher-Yates
  shuffle (i from n-1 down to 1, j = r mod (i+1)) whose r are successive
  outputs of SplitMix64 (Steele, Lea and Flood, 2014) seeded once per call.

Parameter vector (float): W1 (128 x 400, row-major), b1 (128), W2 (128 x 128),
b2 (128), W3 (6 x 128), b3 (6).

``bf16=True`` rounds to bfloat16 (nearest, ties to even) the operands of every
product at the points where a tensor-core implementation keeps them in
bfloat16 (inputs, weight copies, stored activations, back-propagated
pre-activation gradients); everything else stays FP64.  With ``bf16=False``
the network is plain FP64 (the form the finite-difference pins check).
"""
from __future__ import annotations

import math

import numpy as np

N_IN = 387
K_IN = 400
HIDDEN = 128
N_OUT = 6
SHELL_POINTS = 96
SHAPES = [("W1", (HIDDEN, K_IN)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
          ("W3", (N_OUT, HIDDEN)), ("b3", (N_OUT,))]
N_PARAM = sum(int(np.prod(s)) for _, s in SHAPES)
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8

MASK64 = (1 << 64) - 1


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------
def unpack(theta):
    """Views of the flat parameter vector as W1, b1, W2, b2, W3, b3."""
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def init_params(seed):
    """Seeded initial weights (uniform +-1/sqrt(fan_in), zero biases); the
    inputs' padding columns of W1 start at zero."""
    rng = np.random.default_rng(seed)
    th = np.zeros(N_PARAM)
    p = unpack(th)
    for name, fan in (("W1", N_IN), ("W2", HIDDEN), ("W3", HIDDEN)):
        a = 1.0 / math.sqrt(fan)
        p[name][...] = rng.uniform(-a, a, size=p[name].shape)
    p["W1"][:, N_IN:] = 0.0
    return th.astype(np.float32).astype(np.float64)


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = a32.view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (r << 16).astype(np.uint32).view(np.float32).astype(np.float64)


def pad_inputs(X):
    X = np.asarray(X, dtype=np.float64)
    out = np.zeros((X.shape[0], K_IN))
    out[:, :N_IN] = X[:, :N_IN]
    return out


# ---------------------------------------------------------------------------
# forward / backward
# ---------------------------------------------------------------------------
def forward(theta, X, bf=False):
    """Network output for inputs X [n][387 or 400]; returns y and the cache
    the backward pass needs."""
    r = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    p = unpack(np.asarray(theta, dtype=np.float64))
    x = r(pad_inputs(X))
    W1, W2, W3 = r(p["W1"]), r(p["W2"]), r(p["W3"])
    h1 = r(np.tanh(x @ W1.T + p["b1"]))
    h2 = r(np.tanh(h1 @ W2.T + p["b2"]))
    y = h2 @ W3.T + p["b3"]
    return y, dict(x=x, h1=h1, h2=h2, W1=W1, W2=W2, W3=W3)


def loss_and_grad(theta, X, T, bf=False):
    """Mean squared error over the batch and the 6 outputs, and its gradient
    with respect to the parameter vector (back-propagation)."""
    r = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    T = np.asarray(T, dtype=np.float64)
    y, c = forward(theta, X, bf)
    n = y.shape[0]
    d = y - T
    loss = float((d * d).sum() / (n * N_OUT))
    dy = 2.0 * d / (n * N_OUT)
    dyb = r(dy)
    g = np.zeros(N_PARAM)
    gp = unpack(g)
    gp["W3"][...] = dyb.T @ c["h2"]
    gp["b3"][...] = dy.sum(0)
    dz2 = r((dyb @ c["W3"]) * (1.0 - c["h2"] ** 2))
    gp["W2"][...] = dz2.T @ c["h1"]
    gp["b2"][...] = dz2.sum(0)
    dz1 = r((dz2 @ c["W2"]) * (1.0 - c["h1"] ** 2))
    gp["W1"][...] = dz1.T @ c["x"]
    gp["b1"][...] = dz1.sum(0)
    return loss, g


# ---------------------------------------------------------------------------
# SplitMix64 and the batch order
# ---------------------------------------------------------------------------
class SplitMix64:
    """Steele, Lea and Flood (2014): state += 0x9E3779B97F4A7C15, output the
    state mixed by two xor-shift-multiply rounds and a final xor-shift."""

    def __init__(self, seed):
        self.s = int(seed) & MASK64

    def next(self):
        self.s = (self.s + 0x9E3779B97F4A7C15) & MASK64
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)


def shuffle(n, gen):
    perm = list(range(n))
    for i in range(n - 1, 0, -1):
        j = gen.next() % (i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    return np.array(perm, dtype=np.int64)


# ---------------------------------------------------------------------------
# training
# ---------------------------------------------------------------------------
class Adam:
    def __init__(self, n):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0

    def step(self, theta, g, lr):
        self.t += 1
        self.m = ADAM_B1 * self.m + (1 - ADAM_B1) * g
        self.v = ADAM_B2 * self.v + (1 - ADAM_B2) * g * g
        mh = self.m / (1 - ADAM_B1 ** self.t)
        vh = self.v / (1 - ADAM_B2 ** self.t)
        return theta - lr * mh / (np.sqrt(vh) + ADAM_EPS)


def train(theta, X, T, epochs, batch, lr, seed, bf=False, opt=None):
    """Mini-batch Adam; returns the new parameters, the optimiser and the mean
    batch loss of the last epoch."""
    theta = np.array(theta, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    n = X.shape[0]
    opt = opt or Adam(N_PARAM)
    gen = SplitMix64(seed)
    last = 0.0
    for _ in range(epochs):
        perm = shuffle(n, gen)
        losses = []
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            loss, g = loss_and_grad(theta, X[idx], T[idx], bf)
            theta = opt.step(theta, g, lr)
            losses.append(loss)
        last = float(np.mean(losses))
    return theta, opt, last


# ---------------------------------------------------------------------------
# features
# ---------------------------------------------------------------------------
def shell_directions(n=SHELL_POINTS):
    """Fibonacci sphere: z_k = 1 - (2k+1)/n, azimuth k times the golden angle."""
    k = np.arange(n)
    z = 1.0 - (2.0 * k + 1.0) / n
    r = np.sqrt(1.0 - z * z)
    a = k * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([r * np.cos(a), r * np.sin(a), z], axis=1)


def interp_fluid(field, fluid, X):
    """Trilinear interpolation at point X of a periodic [nz][ny][nx] field
    over the fluid corners of the cell (weights renormalised); None when no
    corner is fluid."""
    nz, ny, nx = fluid.shape
    base = np.floor(X).astype(int)
    f = X - base
    acc, wsum = 0.0, 0.0
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = (f[0] if dx else 1 - f[0]) * (f[1] if dy else 1 - f[1]) * (f[2] if dz else 1 - f[2])
                i = ((base[2] + dz) % nz, (base[1] + dy) % ny, (base[0] + dx) % nx)
                if not fluid[i]:
                    continue
                acc = acc + w * field[(Ellipsis,) + i]
                wsum += w
    if wsum <= 0.0:
        return None
    return acc / wsum


def shell_features(phi, u, fluid, xp, vp, wp, R, theta_deg, gap, u_ref, r_ref, box=0.0, wall=False):
    """The 387 inputs of one particle: phi, u: [nz][ny][nx] and [3][nz][ny][nx]
    FP64 fields; fluid: boolean [nz][ny][nx]; xp, vp, wp: centre, velocity,
    angular velocity; R, theta_deg: radius and contact angle.  READING c30:
    with box > 0 each sample is the box filter of width `box` of the fields,
    taken as the mean of the fluid-corner trilinear values at the 3 x 3 x 3
    points (offsets -box/3, 0, +box/3 per axis) of the box around the shell
    point (the midpoint rule of the box average; points whose cell has no
    fluid corner are left out).  With wall (a solid plane z = 0), a point
    whose z lies outside [0, nz) is inside that wall or beyond it and is left
    out too: z is not wrapped across the wall."""
    nz, ny, nx = fluid.shape
    out = np.zeros(N_IN)
    dirs = shell_directions()
    rs = R + gap
    offs = [np.zeros(3)] if box <= 0.0 else [np.array([i, j, k]) * box / 3.0
                                              for k in (-1, 0, 1) for j in (-1, 0, 1) for i in (-1, 0, 1)]
    for k, e in enumerate(dirs):
        phs, us = [], []
        for d in offs:
            X = np.asarray(xp, dtype=np.float64) + rs * e + d
            if wall and not 0.0 <= X[2] < nz:
                continue
            X = np.array([X[0] % nx, X[1] % ny, X[2] % nz])
            p_ = interp_fluid(phi, fluid, X)
            if p_ is None:
                continue
            phs.append(p_)
            us.append(interp_fluid(u, fluid, X))
        if not phs:
            continue
        ph = sum(phs) / len(phs)
        uu = sum(us) / len(us)
        if ph is None:
            continue
        lever = rs * e
        urel = uu - (np.asarray(vp) + np.cross(wp, lever))
        out[4 * k] = ph
        out[4 * k + 1:4 * k + 4] = urel / u_ref
    th = math.radians(theta_deg)
    out[384] = math.cos(th)
    out[385] = math.sin(th)
    out[386] = R / r_ref
    return out
