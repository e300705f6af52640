"""Small case for per-kernel profiler captures (one GPU, a few GB at most).

The drop + spheres workload cropped to 256 x 128 x 64 (2.1 M nodes: the FP32
populations, 320 MB, exceed the L2 size, so DRAM figures stay meaningful),
20 steps to develop the flow, then 3 steps with per-stage event timing
(every kernel launched eagerly, one stream), then one surrogate forward pass
of 4096 rows through the tensor-core GEMMs.  Prints the per-stage times in
microseconds per launch.

    python -m paper_2505_10171_gb300.profile_case fp32
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from paper_2505_10171_gb300 import lbm
from paper_2505_10171_gb300 import workloads as W


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("precision", nargs="?", default="fp32", choices=("fp64", "fp32", "fp16", "bf16"))
    ap.add_argument("--develop", type=int, default=20, help="steps before the timed ones")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--mlp-rows", type=int, default=4096, help="surrogate forward rows (0: none)")
    a = ap.parse_args()
    w = W.cfg2_crop(256, 128, 64)
    c = lbm.Context(dict(w["params"], store_velocity=0), a.precision)
    try:
        if w["particles"]:
            c.lbm_add_particles(w["particles"])
        c.lbm_init_fields(w["phi"])
        c.lbm_step(a.develop)
        c.lbm_profile(1)
        c.lbm_step(a.steps)
        prof = c.lbm_profile_read()
        out = {k: round(v["ms"] / v["launches"] * 1e3, 2) for k, v in prof.items() if v["launches"]}
        if a.mlp_rows > 0:
            rng = np.random.default_rng(5)
            th = (rng.standard_normal(lbm.MLP_PARAMS) * 0.05).astype(np.float32)
            c.lbm_surrogate_load(th)
            X = rng.standard_normal((a.mlp_rows, lbm.MLP_INPUTS)).astype(np.float32)
            Y = c.lbm_surrogate_predict(X)
            out["mlp_rows"] = int(Y.shape[0])
            out["mlp_finite"] = bool(np.isfinite(Y).all())
        print(json.dumps(out))
    finally:
        c.close()


if __name__ == "__main__":
    main()
