"""Pins of the FP64 surrogate oracle (oracle/mlp_oracle.py): back-propagation
against central finite differences, closed forms of the loss and of Adam's
first step, a zero-loss fixed point, the SplitMix64 test vectors, the shuffle,
and the shell sampler on fields whose interpolation is exact."""
import json
import math
import os

import numpy as np
import pytest

from oracle import mlp_oracle as M

GOLD = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.json")


def _data(n, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, M.N_IN)), rng.normal(scale=0.3, size=(n, M.N_OUT))


def test_backprop_matches_central_differences():
    th = M.init_params(3)
    rng = np.random.default_rng(4)
    th = th + rng.normal(scale=0.05, size=th.shape)  # nonzero padding columns and biases too
    X, T = _data(5, 5)
    _, g = M.loss_and_grad(th, X, T)
    offs, o = {}, 0
    for name, shp in M.SHAPES:
        offs[name] = (o, int(np.prod(shp)))
        o += int(np.prod(shp))
    picks = []
    for name, (o, n) in offs.items():
        picks += list(rng.choice(n, size=min(n, 12), replace=False) + o)
    h = 1e-6
    for k in picks:
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (M.loss_and_grad(tp, X, T)[0] - M.loss_and_grad(tm, X, T)[0]) / (2 * h)
        if k >= offs["W1"][0] + 0 and k < offs["b1"][0] and (k - offs["W1"][0]) % M.K_IN >= M.N_IN:
            assert g[k] == 0.0 and abs(fd) < 1e-12  # padding inputs are zero
            continue
        assert abs(fd - g[k]) <= 1e-6 * max(abs(fd), 1e-3), (k, fd, g[k])


def test_loss_and_output_bias_gradient_closed_form():
    """With W3 = 0 the output is b3 for every input: loss = mean (b3 - T)^2
    and dL/db3 = 2 sum_n (b3 - T_n) / (6 n)."""
    th = M.init_params(1)
    p = M.unpack(th)
    p["W3"][...] = 0.0
    p["b3"][...] = np.arange(6) * 0.1 - 0.2
    X, T = _data(7, 2)
    loss, g = M.loss_and_grad(th, X, T)
    d = p["b3"][None, :] - T
    assert abs(loss - (d ** 2).mean()) < 1e-15
    assert np.allclose(M.unpack(g)["b3"], 2 * d.sum(0) / (6 * 7), rtol=0, atol=1e-15)
    assert np.all(M.unpack(g)["W2"] == 0) and np.all(M.unpack(g)["W1"] == 0)  # no path through W3 = 0


def test_adam_first_step_closed_form():
    """Bias correction makes the first step -lr g / (|g| + eps)."""
    rng = np.random.default_rng(0)
    th0 = rng.normal(size=50)
    g = rng.normal(size=50) * 10.0 ** rng.uniform(-6, 1, size=50)
    opt = M.Adam(50)
    th1 = opt.step(th0, g, 1e-3)
    assert np.allclose(th1, th0 - 1e-3 * g / (np.abs(g) + M.ADAM_EPS), rtol=0, atol=1e-15)


def test_teacher_parameters_are_a_stationary_point():
    """Targets made by the network itself: zero loss and a gradient at the
    rounding level on every batch."""
    th = M.init_params(11)
    X, _ = _data(40, 12)
    T, _ = M.forward(th, X)
    for sl in (slice(0, 40), slice(0, 16), slice(16, 40)):
        loss, g = M.loss_and_grad(th, X[sl], T[sl])
        assert loss < 1e-28 and np.abs(g).max() < 1e-14


def test_training_reduces_the_loss_of_a_teacher_problem():
    teacher = M.init_params(21)
    X, _ = _data(256, 22)
    T, _ = M.forward(teacher, X)
    th = M.init_params(23)
    l0 = M.loss_and_grad(th, X, T)[0]
    th, _, last = M.train(th, X, T, epochs=30, batch=64, lr=2e-3, seed=7)
    assert M.loss_and_grad(th, X, T)[0] < 0.1 * l0


def test_splitmix64_published_vectors_and_shuffle():
    gold = json.load(open(GOLD))
    for v in gold["vectors"]:
        g = M.SplitMix64(v["seed"])
        for o in v["outputs"]:
            assert g.next() == int(o, 0)
    perm = M.shuffle(1000, M.SplitMix64(9))
    assert sorted(perm.tolist()) == list(range(1000)) and not np.array_equal(perm, np.arange(1000))
    assert np.array_equal(perm, M.shuffle(1000, M.SplitMix64(9)))


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.140625, 1e-3])
    r = M.bf16(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0  # tie between 1 and 1 + 2^-7: even mantissa (1.0)
    assert r[2] == 1.0 + 2 ** -7  # above the tie
    assert r[3] == -2.5 and r[4] == 3.140625
    assert abs(r[5] - 1e-3) <= 2 ** -9 * 1e-3


def test_shell_directions():
    e = M.shell_directions()
    assert e.shape == (96, 3)
    assert np.allclose(np.linalg.norm(e, axis=1), 1.0, atol=1e-15)
    assert np.allclose(np.diff(e[:, 2]), -2.0 / 96, atol=1e-15) and abs(e[:, 2].sum()) < 1e-12


def test_shell_features_exact_on_linear_and_rigid_fields():
    """Trilinear interpolation is exact for a field linear in x, y, z; the
    relative velocity of a uniform flow past a spinning sphere is
    U - w x (X - x_p) at every point."""
    nx = ny = nz = 32
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    a = np.array([0.011, -0.007, 0.005])
    phi = a[0] * x + a[1] * y + a[2] * z - 0.1
    U0 = np.array([2e-3, -1e-3, 5e-4])
    u = np.stack([np.full(phi.shape, c) for c in U0])
    fluid = np.ones(phi.shape, bool)
    xp, w = np.array([15.3, 16.1, 14.7]), np.array([1e-4, -2e-4, 3e-4])
    R, gap = 5.0, 2.0
    f = M.shell_features(phi, u, fluid, xp, np.zeros(3), w, R, 60.0, gap, 1e-3, 8.0)
    e = M.shell_directions()
    X = xp + (R + gap) * e
    assert np.allclose(f[0:384:4], X @ a - 0.1, rtol=0, atol=1e-14)
    urel = (U0[None, :] - np.cross(w, (R + gap) * e)) / 1e-3
    assert np.allclose(f[1:384:4], urel[:, 0], atol=1e-11)
    assert np.allclose(f[2:384:4], urel[:, 1], atol=1e-11)
    assert np.allclose(f[3:384:4], urel[:, 2], atol=1e-11)
    assert abs(f[384] - 0.5) < 1e-15 and abs(f[385] - math.sqrt(3) / 2) < 1e-15 and f[386] == 5.0 / 8.0
    # reading c30: the box filter's midpoint rule is exact for a linear field,
    # so with a box the linear-field features are unchanged
    fb = M.shell_features(phi, u, fluid, xp, np.zeros(3), w, R, 60.0, gap, 1e-3, 8.0, box=8.0 / 3.0)
    assert np.allclose(fb, f, rtol=0, atol=1e-13)


def test_box_filter_averages_a_quadratic_over_the_box():
    """On phi = x^2 the box filter of width b at X gives the 3-point midpoint
    rule's mean, X^2 + 2 (b/3)^2 / 3 (the grid is coarse enough that the
    trilinear interpolation of x^2 adds (f - f^2) at each sub-point, which
    the reference sums the same way)."""
    n = 40
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    phi = (x.astype(float) - 20.0) ** 2
    u = np.zeros((3, n, n, n))
    fluid = np.ones(phi.shape, bool)
    xp, R, gap, b = np.array([20.2, 19.6, 20.4]), 4.0, 2.0, 2.0
    f = M.shell_features(phi, u, fluid, xp, np.zeros(3), np.zeros(3), R, 90.0, gap, 1e-3, 8.0, box=b)
    e = M.shell_directions()
    X = xp + (R + gap) * e
    want = np.zeros(96)
    for d in (-b / 3, 0.0, b / 3):
        xs = X[:, 0] + d - 20.0
        fr = xs - np.floor(xs)
        want += xs ** 2 + fr * (1.0 - fr)   # linear interpolation of x^2 between nodes
    want /= 3.0
    assert np.allclose(f[0:384:4], want, rtol=0, atol=1e-11)


def test_shell_features_skip_solid_corners():
    """A corner that is not fluid does not enter the interpolation: a field
    that is 7 on fluid and garbage on solid nodes interpolates to 7."""
    n = 24
    phi = np.full((n, n, n), 7.0)
    fluid = np.ones((n, n, n), bool)
    rng = np.random.default_rng(0)
    solid = rng.random((n, n, n)) < 0.3
    phi[solid] = 1e6
    fluid[solid] = False
    u = np.zeros((3, n, n, n))
    f = M.shell_features(phi, u, fluid, np.array([12.0, 12.0, 12.0]), np.zeros(3), np.zeros(3), 4.0, 60.0, 2.0,
                         1e-3, 8.0)
    vals = f[0:384:4]
    seven = np.abs(vals - 7.0) <= 1e-14
    assert np.all(seven | (vals == 0.0))
    assert seven.sum() > 80


def test_shell_features_do_not_reach_across_a_wall():
    """With a solid plane at z = 0 the shell of a sphere resting on it dips
    below the plane; those points read nothing (zero features), while without
    the wall they wrap to the top of the periodic box.  Fields: phi = 1 on the
    lower half of the box, -1 on the upper half, so a wrapped sample would
    read -1 where the sphere's own side of the wall is +1."""
    n = 32
    phi = np.where(np.arange(n)[:, None, None] < n // 2, 1.0, -1.0) * np.ones((n, n, n))
    u = np.zeros((3, n, n, n))
    fluid = np.ones((n, n, n), bool)
    fluid[0] = False  # the wall plane
    xp, R, gap = np.array([16.0, 16.0, 5.0]), 4.0, 2.0
    e = M.shell_directions()
    z = xp[2] + (R + gap) * e[:, 2]
    below = z < 0.0
    assert below.sum() >= 3
    fw = M.shell_features(phi, u, fluid, xp, np.zeros(3), np.zeros(3), R, 90.0, gap, 1e-3, 8.0, wall=True)
    assert np.all(fw[0:384:4][below] == 0.0)
    assert np.all(fw[0:384:4][(z >= 1.0) & (z < n // 2 - 1)] == 1.0)
    fp = M.shell_features(phi, u, fluid, xp, np.zeros(3), np.zeros(3), R, 90.0, gap, 1e-3, 8.0)
    assert np.all(fp[0:384:4][z < -1.0] == -1.0)  # the periodic reading reaches the far side
    # with a box filter, sub-points below the plane are left out of the mean
    fb = M.shell_features(phi, u, fluid, xp, np.zeros(3), np.zeros(3), R, 90.0, gap, 1e-3, 8.0, box=2.0,
                          wall=True)
    assert np.all(fb[0:384:4] >= 0.0)
