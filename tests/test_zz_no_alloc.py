"""The allocation-free mass reduction against lbm_diagnostics (needs a GPU).

lbm_component_masses_noalloc serves callers that cannot call cudaMalloc; it
keeps its scratch in a static device array.  Checked through the C ABI on two
calls in a row, against the context-based reduction, at the FP64 tolerance of
a different summation order.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from helpers import gpu_ctx
from paper_2505_10171_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12


def test_noalloc_masses_match_diagnostics_twice():
    import torch

    from paper_2505_10171_gb300 import build, lbm
    build.build()
    stream = torch.cuda.Stream()
    w = W.cfg1()
    ctx = gpu_ctx(w, "fp64", stream=stream.cuda_stream)
    N = ctx.num_nodes()
    pops = torch.empty(38 * N, dtype=torch.float64, device="cuda")
    masses = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    for steps in (7, 13):
        ctx.lbm_step(steps)
        ref = ctx.lbm_diagnostics()  # synchronises; sums over fluid nodes
        ctx.lbm_read_fields_device(lbm.FIELD_POPS, pops.data_ptr())
        lbm.lbm_component_masses_noalloc(pops.data_ptr(), N, masses.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        got = masses.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert abs(got[0] - ref[0]) <= TOL * abs(ref[0])
        assert abs(got[1] - ref[1]) <= TOL * abs(ref[1])
    ctx.close()


def test_noalloc_rejects_oversized_input():
    from paper_2505_10171_gb300 import lbm
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_component_masses_noalloc(1, (1 << 28) + 1, 1, 0)
    assert e.value.status == lbm.LBM_ERR_ARG
