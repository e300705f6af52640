"""GPU parity of the buoyancy (reading c28): the immersed volume fraction and
the buoyancy force of a sphere half inside a drop, and the trajectory they
drive, against the FP64 oracle."""
import math

import numpy as np
import pytest

from paper_2505_10171_gb300 import lbm
from paper_2505_10171_gb300 import workloads as W
from helpers import gpu_ctx, oracle_sim

pytestmark = pytest.mark.gpu


def immersed_case():
    """The 48x32x32 drop on the sliding wall with its sphere moved to the
    drop's edge (x = 22: the interface crosses the sphere), a weight of 0.02
    and a buoyancy of 1.5 times the weight when fully immersed."""
    w = W.cfg1()
    R = w["particles"][0]["R"]
    vol = 4.0 / 3.0 * math.pi * R ** 3
    w["params"] = dict(w["params"], g_particle=(0.0, 0.0, -0.02), buoyancy_a=(0.0, 0.0, 1.5 * 0.02 / vol))
    w["particles"] = [dict(w["particles"][0], x=(22.0, 16.0, 5.5))]
    return w


def test_buoyancy_matches_oracle_fp64():
    w = immersed_case()
    steps = 60
    o = oracle_sim(w)
    o.step(steps)
    ro = o.particles()[0]
    c = gpu_ctx(w, "fp64")
    c.lbm_step(steps)
    rg = c.lbm_particle_forces()[0]
    c.close()
    assert 0.2 < ro[32] < 0.95  # partly immersed
    assert abs(rg[32] - ro[32]) <= 1e-12
    assert np.abs(rg[33:36] - ro[33:36]).max() <= 1e-12 * np.abs(ro[33:36]).max()
    assert ro[35] > 0.0
    assert np.abs(rg[18:27] - ro[18:27]).max() <= 1e-12


@pytest.mark.parametrize("prec,tol", [("fp16", 2e-3), ("bf16", 2e-3)])
def test_buoyancy_16bit(prec, tol):
    w = immersed_case()
    o = oracle_sim(w)
    o.step(60)
    ro = o.particles()[0]
    c = gpu_ctx(w, prec)
    c.lbm_step(60)
    rg = c.lbm_particle_forces()[0]
    c.close()
    assert abs(rg[32] - ro[32]) <= tol
    assert np.abs(rg[33:36] - ro[33:36]).max() <= tol * np.abs(ro[33:36]).max()


def test_buoyancy_fp32_and_surrogate_guard():
    w = immersed_case()
    steps = 60
    o = oracle_sim(w)
    o.step(steps)
    ro = o.particles()[0]
    c = gpu_ctx(w, "fp32")
    c.lbm_step(steps)
    rg = c.lbm_particle_forces()[0]
    assert abs(rg[32] - ro[32]) <= 1e-4
    # the surrogate replaces the surface sums the buoyancy needs: refused
    from oracle import mlp_oracle as M
    c.lbm_surrogate_load(M.init_params(3))
    with pytest.raises(lbm.LbmError) as e:
        c.lbm_set_force_model(lbm.FORCE_SURROGATE)
    assert e.value.status == 7  # LBM_ERR_UNSUPPORTED
    c.close()
