"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports
every entry point include/lbm.h declares, and the ctypes structs match the C
layout.  No compute call is made (no GPU here)."""
import ctypes as ct
import os
import re
import subprocess
import tempfile

import pytest

from paper_2505_10171_gb300 import build as B
from paper_2505_10171_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_library_exports_every_declared_entry_point(libpath):
    L = ct.CDLL(libpath)
    names = declared_functions()
    assert "lbm_step" in names and "lbm_create" in names and len(names) >= 16
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(lbm.EXPORTS)


def test_binding_loads(libpath):
    L = lbm.load()
    assert L.lbm_last_error(None) == b"null context"
    assert L.lbm_num_nodes(None, 0) == -1


def test_struct_layout_matches_header(libpath):
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "lbm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %d\n", sizeof(lbm_params), offsetof(lbm_params, g_particle),
         offsetof(lbm_params, store_velocity), offsetof(lbm_params, diag_interval), sizeof(lbm_particle),
         offsetof(lbm_particle, theta_deg), offsetof(lbm_particle, kinematic), offsetof(lbm_params, pressure_z),
         offsetof(lbm_params, rho_out), offsetof(lbm_params, buoyancy_a), LBM_PARTICLE_RECORD);
  return 0; }
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    P, Pa = lbm.lbm_params, lbm.lbm_particle
    assert vals == [ct.sizeof(P), P.g_particle.offset, P.store_velocity.offset, P.diag_interval.offset,
                    ct.sizeof(Pa), Pa.theta_deg.offset, Pa.kinematic.offset, P.pressure_z.offset, P.rho_out.offset,
                    P.buoyancy_a.offset, lbm.PARTICLE_RECORD]


def test_abi_velocity_order_matches_header():
    src = open(HEADER).read()
    m = re.search(r"#define LBM_C\s*\\\s*(.*?)\n\n", src, flags=re.S)
    nums = [int(v) for v in re.findall(r"-?\d+", m.group(1).replace("\\", ""))]
    assert nums == lbm.LBM_C.reshape(-1).tolist()


def test_create_without_gpu_fails_cleanly(libpath):
    """With no device, lbm_create reports an error status instead of crashing."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except Exception:
        pass
    with pytest.raises(lbm.LbmError):
        lbm.Context(dict(nx=4, ny=4, nz=4), "fp64")


def test_precision_codes_match_header():
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef enum \{([^}]*)\}\s*lbm_precision;", src).group(1)
    enum = {k: int(v) for k, v in re.findall(r"(LBM_[A-Z0-9_]+)\s*=\s*(\d+)", body)}
    names = {"fp64": "LBM_FP64", "fp32": "LBM_FP32", "fp16": "LBM_FP16_OFFSET", "bf16": "LBM_BF16_OFFSET"}
    assert {k: enum[v] for k, v in names.items()} == lbm.PRECISIONS


BASE = dict(nx=8, ny=8, nz=8)


@pytest.mark.parametrize("bad", [
    dict(nx=0), dict(ny=-3), dict(nx=1024, ny=1024, nz=64),          # sizes; 38 N >= 2^31
    dict(wall_z0=1, nz=2),                                            # a substrate needs 3 planes
    dict(nu_a=0.0), dict(nu_b=float("nan")), dict(rho0=-1.0),
    dict(beta=1.5), dict(sigma=-0.01), dict(theta_wall_deg=180.0),
    dict(wall_velocity=(float("inf"), 0.0, 0.0)), dict(kn=-1.0), dict(mu_r=-0.1),
    dict(cap_norm=-1.0), dict(grad_eps=-1e-4), dict(surrogate_shell_gap=-1.0),
    dict(drop_speed_control=8), dict(drop_speed_interval=-1),
    dict(pressure_z=1, wall_z0=1), dict(pressure_z=1, rho_in=0.0), dict(pressure_z=1, nz=3),
    dict(surrogate_box=-1.0), dict(buoyancy_a=(0.0, 0.0, float("nan"))),
])
def test_create_rejects_invalid_parameters(libpath, bad):
    """Parameters are checked before any device call: an invalid one gives
    LBM_ERR_ARG on any machine, with or without a GPU."""
    with pytest.raises(lbm.LbmError) as e:
        lbm.Context(dict(BASE, **bad), "fp32")
    assert e.value.status == 1  # LBM_ERR_ARG


def test_create_rejects_an_unknown_precision(libpath):
    L = lbm.load()
    arr = (lbm.lbm_params * 1)(lbm.make_params(**BASE))
    h = ct.c_void_p()
    assert L.lbm_create(arr, 1, 9, None, ct.byref(h)) == 7  # LBM_ERR_UNSUPPORTED
    assert L.lbm_create(arr, 1, 4, None, ct.byref(h)) == 7  # the former mixed-storage code
    assert L.lbm_create(arr, 0, 1, None, ct.byref(h)) == 1  # no instances: LBM_ERR_ARG
    assert not h.value


def test_fma_peak_rejects_a_null_output():
    """The FMA microbenchmark checks its argument before touching a device."""
    from paper_2505_10171_gb300 import lbm
    assert lbm.load().lbm_fp32_fma_peak(None) == 1  # LBM_ERR_ARG
