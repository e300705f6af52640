"""Host-side set-up code of the benchmarks and the surrogate campaign (no GPU):
geometry of the detachment and wetting benchmarks, the interface-height
helper, and the resolved / coarse campaign set-ups."""
import math

import numpy as np
import pytest

from paper_2505_10171_gb300 import surrogate_study as SS
from paper_2505_10171_gb300 import validation as V
from paper_2505_10171_gb300 import workloads as W


@pytest.mark.parametrize("theta", [30.0, 90.0, 150.0])
def test_detachment_setup_geometry(theta):
    """The sphere sits at the flat-interface equilibrium height (contact angle
    measured in the liquid below); the liquid layer's order parameter crosses
    zero at z_i = 4 R_p; the pull of 5 R_p stays inside the box."""
    R = 10
    p, phi, part = V.detachment_setup(theta, R)
    nz = p["nz"]
    col = phi.reshape(nz, p["ny"], p["nx"])[:, 0, 0]
    zi = V.interface_height(col)
    assert abs(zi - 4.0 * R) < 1e-9
    assert abs(part["x"][2] - (4.0 * R - R * math.cos(math.radians(theta)))) < 1e-12
    assert part["x"][2] + 5.0 * R + R < nz
    assert part["kinematic"] == 1 and p["wall_z0"] == 0


def test_interface_height_of_a_tanh_profile():
    """Linear interpolation of the zero crossing is exact for an odd profile
    crossing at a node or midway between two, and within 0.03 of the true
    crossing for a tanh of width 2.5 elsewhere (0.07 deg of measured angle at
    R_p = 25)."""
    z = np.arange(100, dtype=np.float64)
    for z0, tol in ((40.0, 1e-12), (40.5, 1e-12), (40.25, 0.03), (61.8, 0.03)):
        col = np.tanh(2.0 * np.minimum(z - 5.0, z0 - z) / W.INTERFACE_WIDTH)
        assert abs(V.interface_height(col) - z0) <= tol


@pytest.mark.parametrize("seed", [1, 7, 101])
def test_campaign_setups_scale_consistently(seed):
    """The coarse set-up is the resolved one at 3/8: box, drop, sphere centres
    in x and y; every sphere keeps a fluid node between itself and the wall
    (delta_R = 1 unscaled, centre R_p + 1.5 above the wall plane) and clear of
    the others by more than the contact distance; sigma, the drop speed and
    the shell (radius 1.5 R_p on either grid) scale as the campaign states;
    only the resolved inputs are box-filtered, over one coarse cell."""
    f, c = SS.resolved(seed), SS.coarse(seed)
    s = SS.SCALE
    pf, pc = f["params"], c["params"]
    assert (pc["nx"], pc["ny"], pc["nz"]) == (96, 48, 48)
    assert abs(pc["sigma"] - pf["sigma"] * s) < 1e-15
    assert abs(pc["drop_speed_target"][0] - pf["drop_speed_target"][0] * s) < 1e-15
    assert pc["delta_R"] == pf["delta_R"] == 1.0
    Rf, Rc_ = f["particles"][0]["R"], c["particles"][0]["R"]
    assert abs(pc["surrogate_shell_gap"] - 0.5 * Rc_) < 1e-12 and abs(pf["surrogate_shell_gap"] - 0.5 * Rf) < 1e-12
    assert pc["surrogate_box"] == 0.0 and abs(pf["surrogate_box"] - 1.0 / s) < 1e-12
    assert all(q["kinematic"] == 1 for q in f["particles"] + c["particles"])  # held spheres
    for qf, qc in zip(f["particles"], c["particles"]):
        assert abs(qc["x"][0] - qf["x"][0] * s) < 1e-12 and abs(qc["x"][1] - qf["x"][1] * s) < 1e-12
        for q, p in ((qf, pf), (qc, pc)):
            assert abs(q["x"][2] - (0.5 + q["R"] + 1.0)) < 1e-12
            # the node plane z = 1 below the centre stays fluid
            assert q["x"][2] - 1.0 > q["R"]
    for ws, p in ((f, pf), (c, pc)):
        xs = np.array([q["x"] for q in ws["particles"]])
        Rc = ws["particles"][0]["R"] + p["delta_R"]
        d = np.linalg.norm(xs[:, None, :2] - xs[None, :, :2], axis=-1) + np.eye(len(xs)) * 1e9
        assert d.min() > 2.0 * Rc
    # damping below the critical value the DEM check accepts
    for ws, p in ((f, pf), (c, pc)):
        R = ws["particles"][0]["R"]
        m = W.PARTICLE_DENSITY * 4.0 / 3.0 * math.pi * R ** 3
        assert 0.0 < p["gn"] < 2.0 * math.sqrt(p["kn"] * m)


def test_resting_damping_is_half_critical():
    for R in (3.0, 8.0):
        m = W.PARTICLE_DENSITY * 4.0 / 3.0 * math.pi * R ** 3
        assert abs(W.resting_damping(R) - math.sqrt(W.COMMON["kn"] * m)) < 1e-12


def test_campaign_smoothing_and_contact_helpers():
    """The moving average keeps a constant series, averages a linear one to
    itself away from the ends, works per sphere, and shortens its window at
    the ends; touching() flags samples whose shell reaches phase a."""
    T, n = 40, 3
    t = np.arange(T, dtype=float)
    Y = np.stack([np.stack([t * (k + 1), np.full(T, 2.0 + k)], axis=1) for k in range(n)], axis=1).reshape(T * n, 2)
    S = SS.smooth(Y, n, 8).reshape(T, n, 2)
    assert np.allclose(S[:, :, 1], 2.0 + np.arange(n))
    # a centred window over 8 samples of a linear series: the mean of t-4 .. t+3
    assert np.allclose(S[10:30, 1, 0], 2.0 * (t[10:30] - 0.5))
    assert np.isclose(S[0, 0, 0], np.mean(t[0:4]))
    assert SS.smooth(Y, n, 1) is Y
    X = np.zeros((3, 387))
    X[0, 0:384:4] = -1.0
    X[1, 0:384:4] = -1.0
    X[1, 40] = 0.2
    X[2, 0:384:4] = 0.9
    assert SS.touching(X).tolist() == [False, True, True]


def test_campaign_contexts_stay_under_the_node_limit():
    ws = [SS.resolved(s) for s in range(1, 26)]
    chunks = SS._chunks(ws)
    assert sorted(i for c in chunks for i in c) == list(range(25))
    for c in chunks:
        assert sum(ws[i]["params"]["nx"] * ws[i]["params"]["ny"] * ws[i]["params"]["nz"] for i in c) <= SS.MAX_NODES
        assert 38 * SS.MAX_NODES < 2 ** 31
    assert max(len(c) for c in chunks) - min(len(c) for c in chunks) <= 1


@pytest.mark.parametrize("seed", [1, 2])
def test_moving_training_spheres_glide_together(seed):
    """Prescribed glide: one velocity for all spheres of a seed, along the
    substrate, scaled with the grid (the angular velocity is the same on both
    grids), rolling without slip on odd seeds; held spheres otherwise."""
    f, c = SS.resolved(seed, moving=True), SS.coarse(seed, moving=True)
    vf = {q["v"] for q in f["particles"]}
    assert len(vf) == 1
    v = np.array(f["particles"][0]["v"])
    assert v[2] == 0.0 and abs(v[0]) <= SS.FINE_U and abs(v[1]) <= SS.FINE_U / 3
    assert np.allclose(np.array(c["particles"][0]["v"]), v * SS.SCALE)
    assert np.allclose(c["particles"][0]["w"], f["particles"][0]["w"])
    w = np.array(f["particles"][0]["w"])
    if seed % 2:
        R = f["particles"][0]["R"]
        assert np.allclose(w, [-v[1] / R, v[0] / R, 0.0])
    else:
        assert np.all(w == 0.0)
    assert all(q["kinematic"] == 1 for q in f["particles"])
    assert "v" not in SS.resolved(seed)["particles"][0]
