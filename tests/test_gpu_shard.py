"""The sharded batch on the GPU: each rank's share stepped in its own context
gives, per instance, the bits of the whole batch in one context (instances
are independent).  Both shares of a two-rank split run here one after the
other on the same GPU; no collective is involved."""
import numpy as np
import pytest

from paper_2505_10171_gb300 import shard
from paper_2505_10171_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _small_batch():
    out = []
    for k, (nx, ny, nz, R) in enumerate(((48, 24, 20, 7.0), (40, 28, 18, 6.0), (32, 24, 24, 5.0))):
        p = dict(W.COMMON, nx=nx, ny=ny, nz=nz, wall_z0=1, theta_wall_deg=80.0 + 10 * k, nu_a=1 / 6, nu_b=1 / 30)
        phi = W.drop_phi(nx, ny, nz, (nx / 3, ny / 2, 0.5), R)
        parts = [dict(x=(nx / 3 + R + 6.0, ny / 2, 4.5), R=3.0, theta_deg=90.0, rho_p=W.PARTICLE_DENSITY)]
        out.append(dict(params=p, phi=phi, particles=parts))
    return out


def test_two_rank_shares_equal_the_whole_batch():
    ws = _small_batch()
    whole = shard.run_shard(ws, 12, "fp32", 0, 1)
    parts = {}
    for rank in range(2):
        parts.update(shard.run_shard(ws, 12, "fp32", rank, 2))
    assert sorted(parts) == sorted(whole) == [0, 1, 2]
    for k in whole:
        assert np.array_equal(parts[k][0], whole[k][0])
        assert np.array_equal(parts[k][1][:2], whole[k][1][:2])
