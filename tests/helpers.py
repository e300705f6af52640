"""Shared test helpers: build the oracle and the CUDA context from one workload dict."""
import numpy as np

def oracle_sim(w):
    import oracle as O
    return O.from_workload(w)


def gpu_ctx(w, precision="fp64", store_velocity=True, stream=None):
    from paper_2505_10171_gb300 import lbm
    p = dict(w["params"])
    p["store_velocity"] = 1 if store_velocity else 0
    c = lbm.Context(p, precision, stream=stream)
    if w.get("mask") is not None:
        c.lbm_set_solid_mask(w["mask"])
    if w.get("particles"):
        c.lbm_add_particles(w["particles"])
    c.lbm_init_fields(w["phi"], w.get("rho"), w.get("u"))
    return c


def rel_l2(a, b):
    a, b = np.asarray(a, dtype=np.float64).ravel(), np.asarray(b, dtype=np.float64).ravel()
    d = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (d if d > 0 else 1.0)
