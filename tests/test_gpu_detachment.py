"""Benchmarks of the method on the GPU.  Capillary detachment (Sec. V G): the largest capillary
force on a sphere pulled out of a flat interface at v_p = 0.01 against
Scheludko's F_max = 2 pi sigma R_p cos^2(theta_p / 2).  The paper reports
agreement within 5% at R_p = 25 and errors up to 30% at R_p = 10; the bands
below are those."""
import numpy as np
import pytest

from paper_2505_10171_gb300 import validation as V

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("theta", [110.0])
def test_detachment_force_large_sphere(theta):
    r = V.detachment(theta, R_p=25)
    print(theta, r["F_max"], r["F_pred"], r["ratio"])
    assert abs(r["ratio"] - 1.0) <= 0.05
    # the force opposes the pull and peaks before the sphere has left the interface
    assert r["Fz"][0] < 0.0 and 0.2 < r["t_at_max"] < 4.5


@pytest.mark.parametrize("theta", [50.0, 90.0, 130.0])
def test_detachment_force_small_sphere(theta):
    r = V.detachment(theta, R_p=10)
    print(theta, r["ratio"])
    assert abs(r["ratio"] - 1.0) <= 0.3


def test_wetting_equilibrium_large_sphere():
    """Sec. V E particle-at-interface benchmark: a free sphere released on a
    flat interface settles at the height that gives its contact angle."""
    r = V.wetting_equilibrium(110.0, R_p=25)
    print(r["theta_mes"], r["z_i"], r["z_c"][-1])
    assert abs(r["theta_mes"] - 110.0) <= 5.0


@pytest.mark.parametrize("theta", [70.0, 130.0])
def test_wetting_equilibrium_small_sphere(theta):
    """The paper reports discrepancies up to about 16% for its worst cases."""
    r = V.wetting_equilibrium(theta, R_p=10)
    print(theta, r["theta_mes"])
    assert abs(r["theta_mes"] - theta) <= 0.16 * theta


def test_tube_migration_drifts_outward():
    """The off-axis sphere in Poiseuille flow drifts away from the axis
    (l / R_t = 0.3 lies inside the Segre-Silberberg equilibrium near 0.6),
    steadily, and the flow far from the sphere keeps the centreline speed
    within 5%.  (Once the drift is steady its mean lateral force is zero: the
    lift is balanced by the drag on the radial motion.)"""
    r = V.tube_migration(nz=256, steps=6000, sample_every=200)
    print(r["l"][::5], r["u_axis"])
    assert r["l"][-1] > r["l"][0]
    assert np.all(np.diff(r["l"][len(r["l"]) // 3:]) > 0.0)
    assert abs(r["u_axis"] / 0.02 - 1.0) < 0.05
