"""ctypes binding of the C ABI in include/lbm.h (argument marshalling only).

Every function here forwards to the entry point of the same name in
``_lib/liblbm.so``; all computation runs in the CUDA kernels behind it.  There
is no CPU fallback: loading fails loudly when the library is missing.

Arrays follow the ABI layout: z-major fields, vector fields as [3][N],
populations f^a then f^b as [38][N] in the LBM_C velocity order.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liblbm.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_STATE, LBM_ERR_UNSTABLE, LBM_ERR_TIMEOUT, \
    LBM_ERR_UNSUPPORTED = range(8)
STATUS_NAMES = ["LBM_OK", "LBM_ERR_ARG", "LBM_ERR_OOM", "LBM_ERR_CUDA", "LBM_ERR_STATE", "LBM_ERR_UNSTABLE",
                "LBM_ERR_TIMEOUT", "LBM_ERR_UNSUPPORTED"]
# storage of the total offsets F; the per-node order parameter, recolouring
# amplitude and normal are FP64 in the FP64 form and FP32 otherwise
PRECISIONS = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}
FIELD_RHO_A, FIELD_RHO_B, FIELD_PHI, FIELD_U, FIELD_POPS, FIELD_OWNER = 1, 2, 4, 8, 16, 32
PARTICLE_RECORD = 36
PARTICLE_STATE = 19
MAX_PARTICLES = 61
# velocity order of population arrays at the ABI (LBM_C)
LBM_C = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 0],
                  [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1], [0, 1, 1],
                  [0, -1, -1], [0, 1, -1], [0, -1, 1]], dtype=np.int32)


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class lbm_params(ct.Structure):
    _fields_ = [
        ("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
        ("wall_z0", ct.c_int),
        ("wall_velocity", ct.c_double * 3),
        ("theta_wall_deg", ct.c_double),
        ("rho0", ct.c_double),
        ("nu_a", ct.c_double), ("nu_b", ct.c_double),
        ("sigma", ct.c_double), ("beta", ct.c_double), ("cap_norm", ct.c_double),
        ("body_force_a", ct.c_double * 3), ("body_force_b", ct.c_double * 3),
        ("kn", ct.c_double), ("kt", ct.c_double), ("kr", ct.c_double),
        ("gn", ct.c_double), ("gt", ct.c_double), ("gr", ct.c_double),
        ("mu_s", ct.c_double), ("mu_r", ct.c_double), ("delta_R", ct.c_double),
        ("g_particle", ct.c_double * 3),
        ("grad_eps", ct.c_double), ("wet_phi_max", ct.c_double),
        ("store_velocity", ct.c_int), ("diag_interval", ct.c_int),
        ("surrogate_u_ref", ct.c_double), ("surrogate_r_ref", ct.c_double), ("surrogate_shell_gap", ct.c_double),
        ("drop_speed_control", ct.c_int), ("drop_speed_target", ct.c_double * 3),
        ("drop_speed_kp", ct.c_double), ("drop_speed_ki", ct.c_double), ("drop_speed_interval", ct.c_int),
        ("pressure_z", ct.c_int), ("rho_in", ct.c_double), ("rho_out", ct.c_double),
        ("surrogate_box", ct.c_double),
        ("buoyancy_a", ct.c_double * 3),
    ]


class lbm_particle(ct.Structure):
    _fields_ = [
        ("x", ct.c_double * 3), ("v", ct.c_double * 3), ("w", ct.c_double * 3),
        ("R_p", ct.c_double), ("rho_p", ct.c_double), ("theta_deg", ct.c_double),
        ("kinematic", ct.c_int),
    ]


_lib = None
EXPORTS = ["lbm_create", "lbm_destroy", "lbm_last_error", "lbm_set_solid_mask", "lbm_init_fields",
           "lbm_init_fields_device", "lbm_add_particles", "lbm_step", "lbm_particle_forces", "lbm_read_fields",
           "lbm_read_fields_device", "lbm_num_particles", "lbm_num_nodes", "lbm_diagnostics",
           "lbm_last_launch_count", "lbm_profile", "lbm_profile_read", "lbm_component_masses_noalloc",
           "lbm_set_fluid_kernel", "lbm_fluid_form_in_use", "lbm_set_force_model", "lbm_surrogate_load",
           "lbm_surrogate_save", "lbm_surrogate_predict", "lbm_surrogate_gradient", "lbm_surrogate_train",
           "lbm_surrogate_features", "lbm_drop_speed_state", "lbm_autotune", "lbm_set_particle_motion",
           "lbm_inject_fault", "lbm_particle_state_size", "lbm_get_particle_state", "lbm_set_particle_state",
           "lbm_run_state_size", "lbm_get_run_state", "lbm_set_run_state", "lbm_particle_forces_async",
           "lbm_set_record_ring", "lbm_fp32_fma_peak"]
# learned force surrogate (include/lbm.h)
MLP_INPUTS, MLP_OUTPUTS, MLP_PARAMS, MLP_MAX_BATCH = 387, 6, 68614, 4096
FORCE_RESOLVED, FORCE_SURROGATE = 0, 1
FAULT_NONE, FAULT_GEMM_NO_COMMIT = 0, 1
STAGES = ["phi", "solid_phi", "grad_wetting", "collide", "momentum_exchange", "capillary", "dem", "geom_owner",
          "geom_boundary", "refill", "fused", "particle_region", "curvature", "surrogate", "phi_boundary",
          "collide_boundary"]
# the launch form of lbm_set_fluid_kernel
FORM_PLAIN = 2


def load(path: str = LIB_PATH):
    """Load liblbm.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ct.CDLL(path)
    P, d, i, vp = ct.POINTER, ct.POINTER(ct.c_double), ct.c_int, ct.c_void_p
    L.lbm_create.argtypes = [P(lbm_params), i, i, vp, P(vp)]
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_last_error.argtypes = [vp]
    L.lbm_last_error.restype = ct.c_char_p
    L.lbm_set_solid_mask.argtypes = [vp, i, P(ct.c_uint8)]
    L.lbm_init_fields.argtypes = [vp, i, d, d, d, d]
    L.lbm_init_fields_device.argtypes = [vp, i, vp, vp, vp]
    L.lbm_add_particles.argtypes = [vp, i, i, P(lbm_particle)]
    L.lbm_step.argtypes = [vp, i]
    L.lbm_particle_forces.argtypes = [vp, i, d]
    L.lbm_particle_forces_async.argtypes = [vp, i, d]
    L.lbm_set_record_ring.argtypes = [vp, vp, i]
    L.lbm_fp32_fma_peak.argtypes = [d]
    L.lbm_set_particle_motion.argtypes = [vp, i, i, d, d]
    L.lbm_read_fields.argtypes = [vp, i, ct.c_uint, d]
    L.lbm_read_fields_device.argtypes = [vp, i, ct.c_uint, vp]
    L.lbm_num_particles.argtypes = [vp, i]
    L.lbm_num_particles.restype = i
    L.lbm_num_nodes.argtypes = [vp, i]
    L.lbm_num_nodes.restype = ct.c_longlong
    L.lbm_diagnostics.argtypes = [vp, i, d]
    L.lbm_fluid_form_in_use.argtypes = [vp]
    L.lbm_fluid_form_in_use.restype = i
    L.lbm_last_launch_count.argtypes = [vp]
    L.lbm_last_launch_count.restype = ct.c_longlong
    L.lbm_particle_state_size.argtypes = [vp, i]
    L.lbm_particle_state_size.restype = ct.c_longlong
    L.lbm_run_state_size.argtypes = [vp]
    L.lbm_run_state_size.restype = ct.c_longlong
    L.lbm_profile.argtypes = [vp, i]
    L.lbm_profile_read.argtypes = [vp, d, i]
    L.lbm_component_masses_noalloc.argtypes = [vp, ct.c_longlong, vp, vp]
    L.lbm_set_fluid_kernel.argtypes = [vp, i, i, i]
    fp = ct.POINTER(ct.c_float)
    sz = ct.c_size_t
    L.lbm_set_force_model.argtypes = [vp, i]
    L.lbm_surrogate_load.argtypes = [vp, fp, sz]
    L.lbm_surrogate_save.argtypes = [vp, fp, sz]
    L.lbm_surrogate_predict.argtypes = [vp, fp, sz, fp]
    L.lbm_surrogate_gradient.argtypes = [vp, fp, fp, sz, fp, d]
    L.lbm_surrogate_train.argtypes = [vp, fp, fp, sz, i, i, ct.c_double, ct.c_uint64, d]
    L.lbm_surrogate_features.argtypes = [vp, i, fp]
    L.lbm_drop_speed_state.argtypes = [vp, i, d]
    L.lbm_autotune.argtypes = [vp, i, P(ct.c_int), P(ct.c_int), d]
    L.lbm_inject_fault.argtypes = [vp, i]
    L.lbm_get_particle_state.argtypes = [vp, i, d, ct.c_size_t]
    L.lbm_get_run_state.argtypes = [vp, d, ct.c_size_t]
    L.lbm_set_run_state.argtypes = [vp, d, ct.c_size_t]
    L.lbm_set_particle_state.argtypes = [vp, i, d, ct.c_size_t]
    for name in EXPORTS:
        if name not in ("lbm_destroy", "lbm_last_error", "lbm_num_particles", "lbm_num_nodes",
                        "lbm_last_launch_count", "lbm_particle_state_size", "lbm_run_state_size"):
            getattr(L, name).restype = ct.c_int
    _lib = L
    return L


PARAM_DEFAULTS = dict(
    wall_z0=0, wall_velocity=(0.0, 0.0, 0.0), theta_wall_deg=90.0, rho0=1.0, nu_a=1.0 / 6.0, nu_b=1.0 / 6.0,
    sigma=0.01, beta=0.7, cap_norm=0.0, body_force_a=(0.0, 0.0, 0.0), body_force_b=(0.0, 0.0, 0.0), kn=2.5,
    kt=1.0, kr=0.5, gn=0.0, gt=0.0, gr=0.0, mu_s=0.0, mu_r=0.0, delta_R=1.0, g_particle=(0.0, 0.0, 0.0),
    grad_eps=0.0, wet_phi_max=0.0, store_velocity=0, diag_interval=0,
    surrogate_u_ref=0.0, surrogate_r_ref=0.0, surrogate_shell_gap=0.0,
    drop_speed_control=0, drop_speed_target=(0.0, 0.0, 0.0), drop_speed_kp=0.0, drop_speed_ki=0.0,
    drop_speed_interval=0, pressure_z=0, rho_in=1.0, rho_out=1.0, surrogate_box=0.0,
    buoyancy_a=(0.0, 0.0, 0.0),
)


def make_params(**kw) -> lbm_params:
    v = dict(PARAM_DEFAULTS)
    v.update({k: val for k, val in kw.items() if k in lbm_params.__dict__ or k in PARAM_DEFAULTS or
              k in ("nx", "ny", "nz")})
    p = lbm_params()
    for name, typ in lbm_params._fields_:
        val = v[name]
        if isinstance(val, (tuple, list, np.ndarray)):
            arr = getattr(p, name)
            for k in range(3):
                arr[k] = float(val[k])
        else:
            setattr(p, name, int(val) if typ is ct.c_int else float(val))
    return p


def lbm_component_masses_noalloc(pops_ptr, n_nodes, masses_ptr, stream=0):
    """FP64 sums of f^a and f^b of a device population array ([38][n_nodes],
    ABI layout) into a device buffer of 2 doubles, without any allocation."""
    st = load().lbm_component_masses_noalloc(ct.c_void_p(pops_ptr), int(n_nodes), ct.c_void_p(masses_ptr),
                                             ct.c_void_p(stream or 0))
    if st != LBM_OK:
        raise LbmError(st, "lbm_component_masses_noalloc failed")


def lbm_fp32_fma_peak():
    """Measured FP32 multiply-add throughput of the current device, TFLOP/s."""
    out = ct.c_double(0.0)
    st = load().lbm_fp32_fma_peak(ct.byref(out))
    if st != LBM_OK:
        raise LbmError(st, "lbm_fp32_fma_peak failed")
    return out.value


def _dp(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _fp(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_float))


class Context:
    """An lbm_ctx of one or more instances; methods mirror the C entry points."""

    def __init__(self, params, precision="fp64", stream=None):
        self.L = load()
        plist = params if isinstance(params, (list, tuple)) else [params]
        arr = (lbm_params * len(plist))(*[make_params(**p) if isinstance(p, dict) else p for p in plist])
        self.params = arr
        self.n_inst = len(plist)
        h = ct.c_void_p()
        st = self.L.lbm_create(arr, len(plist), PRECISIONS[precision], ct.c_void_p(stream or 0), ct.byref(h))
        if st != LBM_OK:
            raise LbmError(st, "lbm_create failed")
        self.h = h
        self.precision = precision

    def _check(self, st):
        if st != LBM_OK:
            raise LbmError(st, self.L.lbm_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_nodes(self, inst=0):
        return int(self.L.lbm_num_nodes(self.h, inst))

    def num_particles(self, inst=0):
        return int(self.L.lbm_num_particles(self.h, inst))

    # --- entry points -------------------------------------------------------
    def lbm_set_solid_mask(self, mask, inst=0):
        m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        self._check(self.L.lbm_set_solid_mask(self.h, inst, m.ctypes.data_as(ct.POINTER(ct.c_uint8))))

    def lbm_init_fields(self, phi=None, rho=None, u=None, pops=None, inst=0):
        arrs = [None if a is None else _f64(a).reshape(-1) for a in (phi, rho, u, pops)]
        ptr = [ct.cast(None, ct.POINTER(ct.c_double)) if a is None else _dp(a) for a in arrs]
        self._check(self.L.lbm_init_fields(self.h, inst, *ptr))

    def lbm_init_fields_device(self, phi_ptr, rho_ptr=0, u_ptr=0, inst=0):
        self._check(self.L.lbm_init_fields_device(self.h, inst, ct.c_void_p(phi_ptr), ct.c_void_p(rho_ptr or 0),
                                                  ct.c_void_p(u_ptr or 0)))

    def lbm_add_particles(self, parts, inst=0):
        arr = (lbm_particle * max(1, len(parts)))()
        for k, q in enumerate(parts):
            for name in ("x", "v", "w"):
                vals = q.get(name, (0.0, 0.0, 0.0))
                for a in range(3):
                    getattr(arr[k], name)[a] = float(vals[a])
            arr[k].R_p = float(q["R"])
            arr[k].rho_p = float(q.get("rho_p", 0.125))
            arr[k].theta_deg = float(q.get("theta_deg", 90.0))
            arr[k].kinematic = int(q.get("kinematic", 0))
        self._check(self.L.lbm_add_particles(self.h, inst, len(parts), arr))

    def lbm_step(self, n=1):
        self._check(self.L.lbm_step(self.h, int(n)))

    def lbm_set_particle_motion(self, p, v, w=(0.0, 0.0, 0.0), inst=0):
        """Velocity and angular velocity of particle p (prescribed motion of a
        kinematic particle), applied from the next step on."""
        v = np.ascontiguousarray(v, dtype=np.float64)
        w = np.ascontiguousarray(w, dtype=np.float64)
        self._check(self.L.lbm_set_particle_motion(self.h, inst, int(p), _dp(v), _dp(w)))

    def lbm_particle_forces(self, inst=0, out=None):
        n = self.num_particles(inst)
        out = np.zeros((max(n, 1), PARTICLE_RECORD)) if out is None else out
        self._check(self.L.lbm_particle_forces(self.h, inst, _dp(out)))
        return out[:n]

    def lbm_get_particle_state(self, inst=0):
        """The particles' checkpoint (include/lbm.h): LBM_PARTICLE_STATE
        doubles per particle, then the friction-spring histories."""
        n = int(self.L.lbm_particle_state_size(self.h, inst))
        if n < 0:
            raise LbmError(1, "bad instance")
        out = np.zeros(max(n, 1))
        self._check(self.L.lbm_get_particle_state(self.h, inst, _dp(out), ct.c_size_t(n)))
        return out[:n]

    def lbm_set_particle_state(self, state, inst=0):
        st = np.ascontiguousarray(state, dtype=np.float64)
        self._check(self.L.lbm_set_particle_state(self.h, inst, _dp(st), ct.c_size_t(st.size)))

    def lbm_get_run_state(self):
        """Steps taken, then per instance the phase-a body force, the
        drop-speed control's error integral and last measured velocity."""
        n = int(self.L.lbm_run_state_size(self.h))
        out = np.zeros(n)
        self._check(self.L.lbm_get_run_state(self.h, _dp(out), ct.c_size_t(n)))
        return out

    def lbm_set_run_state(self, state):
        st = np.ascontiguousarray(state, dtype=np.float64)
        self._check(self.L.lbm_set_run_state(self.h, _dp(st), ct.c_size_t(st.size)))

    def lbm_particle_forces_async(self, out, inst=0):
        """Enqueue the read of the particle records into out (a float64 array of
        at least n_particles x PARTICLE_RECORD; page-locked memory is written by
        the device directly, pageable memory through a copy); valid after the
        next synchronisation."""
        n = self.num_particles(inst)
        if out.dtype != np.float64 or not out.flags.c_contiguous or out.size < n * PARTICLE_RECORD:
            raise ValueError("out must be a C-contiguous float64 array of n_particles x PARTICLE_RECORD")
        self._check(self.L.lbm_particle_forces_async(self.h, inst, _dp(out)))

    def lbm_set_record_ring(self, ring):
        """Record every step's particle records (all instances) into ring, a
        float64 array of slots x n_particles_total x PARTICLE_RECORD in
        page-locked host memory (or a device tensor's pointer given as an int
        with its slot count: (ptr, slots)); step k since the call goes to slot
        k mod slots.  None stops the recording."""
        if ring is None:
            self._ring = None
            self._check(self.L.lbm_set_record_ring(self.h, None, 0))
            return
        if isinstance(ring, tuple):
            ptr, slots = ring
            self._check(self.L.lbm_set_record_ring(self.h, ct.c_void_p(int(ptr)), int(slots)))
            self._ring = ring
            return
        if ring.dtype != np.float64 or not ring.flags.c_contiguous or ring.ndim < 2:
            raise ValueError("ring must be a C-contiguous float64 array of slots x records")
        self._check(self.L.lbm_set_record_ring(self.h, ring.ctypes.data_as(ct.c_void_p), int(ring.shape[0])))
        self._ring = ring

    def lbm_read_fields(self, mask, inst=0, out=None):
        N = self.num_nodes(inst)
        cnt = sum(c for bit, c in ((1, 1), (2, 1), (4, 1), (8, 3), (16, 38), (32, 1)) if mask & bit)
        out = np.zeros(cnt * N) if out is None else out
        self._check(self.L.lbm_read_fields(self.h, inst, int(mask), _dp(out)))
        return out

    def lbm_read_fields_device(self, mask, out_ptr, inst=0):
        self._check(self.L.lbm_read_fields_device(self.h, inst, int(mask), ct.c_void_p(out_ptr)))

    def lbm_diagnostics(self, inst=0):
        out = np.zeros(4)
        self._check(self.L.lbm_diagnostics(self.h, inst, _dp(out)))
        return out

    def lbm_set_fluid_kernel(self, form=FORM_PLAIN, tile=0, zchunk=0):
        self._check(self.L.lbm_set_fluid_kernel(self.h, int(form), int(tile), int(zchunk)))

    def lbm_fluid_form_in_use(self):
        return int(self.L.lbm_fluid_form_in_use(self.h))

    def lbm_last_launch_count(self):
        return int(self.L.lbm_last_launch_count(self.h))

    def lbm_profile(self, enable=True):
        self._check(self.L.lbm_profile(self.h, int(enable)))

    def lbm_profile_read(self):
        out = np.zeros(2 * len(STAGES))
        self._check(self.L.lbm_profile_read(self.h, _dp(out), len(STAGES)))
        return {name: dict(launches=int(out[2 * k]), ms=float(out[2 * k + 1])) for k, name in enumerate(STAGES)}

    def lbm_autotune(self, steps=20):
        """(tile, z-chunk per instance, ms per step of the chosen shape)."""
        t = ct.c_int()
        zc = (ct.c_int * self.n_inst)()
        ms = np.zeros(1)
        self._check(self.L.lbm_autotune(self.h, int(steps), ct.byref(t), zc, _dp(ms)))
        return t.value, list(zc), float(ms[0])

    def lbm_inject_fault(self, fault):
        self._check(self.L.lbm_inject_fault(self.h, int(fault)))

    def lbm_drop_speed_state(self, inst=0):
        out = np.zeros(6)
        self._check(self.L.lbm_drop_speed_state(self.h, inst, _dp(out)))
        return out[:3], out[3:]

    # --- learned force surrogate --------------------------------------------
    def lbm_set_force_model(self, model):
        self._check(self.L.lbm_set_force_model(self.h, int(model)))

    def lbm_surrogate_load(self, weights):
        w = _f32(weights)
        self._check(self.L.lbm_surrogate_load(self.h, _fp(w), w.size))

    def lbm_surrogate_save(self):
        w = np.zeros(MLP_PARAMS, dtype=np.float32)
        self._check(self.L.lbm_surrogate_save(self.h, _fp(w), w.size))
        return w

    def lbm_surrogate_predict(self, X):
        X = _f32(X).reshape(-1, MLP_INPUTS)
        Y = np.zeros((X.shape[0], MLP_OUTPUTS), dtype=np.float32)
        self._check(self.L.lbm_surrogate_predict(self.h, _fp(X), X.shape[0], _fp(Y)))
        return Y

    def lbm_surrogate_gradient(self, X, Y):
        X = _f32(X).reshape(-1, MLP_INPUTS)
        Y = _f32(Y).reshape(-1, MLP_OUTPUTS)
        g = np.zeros(MLP_PARAMS, dtype=np.float32)
        loss = np.zeros(1)
        self._check(self.L.lbm_surrogate_gradient(self.h, _fp(X), _fp(Y), X.shape[0], _fp(g), _dp(loss)))
        return g, float(loss[0])

    def lbm_surrogate_train(self, X, Y, epochs, batch, lr, seed):
        X = _f32(X).reshape(-1, MLP_INPUTS)
        Y = _f32(Y).reshape(-1, MLP_OUTPUTS)
        loss = np.zeros(1)
        self._check(self.L.lbm_surrogate_train(self.h, _fp(X), _fp(Y), X.shape[0], int(epochs), int(batch),
                                               float(lr), ct.c_uint64(int(seed) & (2 ** 64 - 1)), _dp(loss)))
        return float(loss[0])

    def lbm_surrogate_features(self, inst=0):
        n = self.num_particles(inst)
        out = np.zeros((max(n, 1), MLP_INPUTS), dtype=np.float32)
        self._check(self.L.lbm_surrogate_features(self.h, inst, _fp(out)))
        return out[:n]

    # --- conveniences built only from the entry points above ----------------
    def fields(self, inst=0):
        """rho_a, rho_b, phi (and u when stored) of an instance as a dict."""
        N = self.num_nodes(inst)
        p = self.params[inst]
        mask = FIELD_RHO_A | FIELD_RHO_B | FIELD_PHI | (FIELD_U if p.store_velocity else 0)
        out = self.lbm_read_fields(mask, inst)
        d = dict(rho_a=out[:N], rho_b=out[N:2 * N], phi=out[2 * N:3 * N])
        if p.store_velocity:
            d["u"] = out[3 * N:6 * N].reshape(3, N)
        return d

    def pops(self, inst=0):
        N = self.num_nodes(inst)
        out = self.lbm_read_fields(FIELD_POPS, inst).reshape(38, N)
        return out[:19], out[19:]

    def owner(self, inst=0):
        return self.lbm_read_fields(FIELD_OWNER, inst).astype(np.uint8)
