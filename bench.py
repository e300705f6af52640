#!/usr/bin/env python
"""Benchmark of the coupled LBM-DEM time step on GB300.

One "step" is one coupled time step of the whole hot path (streaming with
bounce-back, order parameter, gradient with wetting, curvature and CSF force,
MRT collision with Guo forcing, recolouring, momentum exchange, capillary
force, DEM, geometry update and refill) over the 256x128x128 drop + 8 spheres
workload (FP32 offset storage).  The metric is MLUPS (all nodes x steps /
time).  Inputs are synthetic (seeded), see paper_2505_10171_gb300/workloads.py.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Under torchrun each rank steps its own copy
of the workload (independent problems, weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline at 1 GB300 (FP32 vs FP16-storage vs batched) at stated error"
UNIT = "MLUPS"
WORKLOAD = "drop R=40 sliding over a 150 deg wall + 8 spheres R_p=8, 256x128x128 (4.19M nodes), coupled LBM-DEM step"
# bytes of one stored total population (F) and of one per-node real (phi, b,
# normal, |grad phi|, curvature)
ELEM = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}
REAL = {"fp64": 8, "fp32": 4, "fp16": 4, "bf16": 4}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16": "f16-storage/f32-math", "bf16": "bf16-storage/f32-math"}


def method_bytes_per_lu(prec):
    """The method's population traffic per lattice update: read and write of
    2 x 19 populations at the storage precision."""
    return 2 * 38 * ELEM[prec]


def population_bytes_per_node(stage, prec):
    """Population bytes a kernel moves per node: the order-parameter pass reads
    the 19 streamed total populations, the collision reads them again and
    writes 19."""
    e = ELEM[prec]
    return {"collide": 38 * e, "phi": 19 * e}.get(stage, 0)


def design_bytes_per_node(stage, prec):
    """Every byte a kernel reads or writes per node, each once: populations
    plus the per-node reals (phi, the colour record of 4 reals, n,
    |grad phi|, kappa), flags left out.  Order parameter: 19 F + the sources'
    records + phi out; gradient pass: phi in, n, |grad phi|, kappa out;
    collision: 19 F + phi, n, |grad phi|, kappa in, 19 F + record out."""
    e, r = ELEM[prec], REAL[prec]
    return {"phi": 19 * e + 5 * r, "grad_wetting": 6 * r, "collide": 38 * e + 10 * r}.get(stage, 0)


# dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant
# kernel, from one ncu --set full capture of the 256x128x64 crop of the
# workload (python -m paper_2505_10171_gb300.profile_case fp32), scaled by
# the node count to the 256x128x128 launch (traffic grows with the nodes);
# valid only for the fluid-kernel sources it was taken on (their hash)
NCU_TRAFFIC = {("collide", "fp32"): (2 * 348004096, "569acf308faaf088")}
FLUID_SOURCES = ("paper_2505_10171_gb300/csrc/lbm_fluid.cu", "paper_2505_10171_gb300/csrc/lbm_node.cuh",
                 "paper_2505_10171_gb300/csrc/lbm_internal.cuh")


def fluid_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in FLUID_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(stage, prec):
    v = NCU_TRAFFIC.get((stage, prec))
    return v[0] if v and v[1] == fluid_source_hash() else None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def omp_threads(n):
    """Threads of the oracle's OpenMP loops from now on (its libgomp is the
    process's); returns the count set, or None if libgomp is not loadable."""
    import ctypes
    try:
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(int(n))
        return int(n)
    except OSError:
        return None


def oracle_sample(budget_s=15.0, steps_cap=None, threads=None):
    """Time the FP64 CPU oracle on a sub-box of the workload (host cores; all
    of them, or `threads`)."""
    import oracle as O
    from paper_2505_10171_gb300 import workloads as W
    O.lib()
    cores = omp_threads(threads if threads else os.cpu_count()) or os.cpu_count()
    for dims in ((128, 128, 48), (96, 96, 40), (64, 64, 32)):
        w = W.cfg2_crop(*dims)
        s = O.from_workload(w)
        t0 = time.perf_counter()
        s.step(1)
        t1 = time.perf_counter() - t0
        if t1 * 3 <= budget_s or dims == (64, 64, 32):
            break
    n = max(1, int(budget_s / max(t1, 1e-3)))
    if steps_cap:
        n = min(n, steps_cap)
    t0 = time.perf_counter()
    s.step(n)
    dt = time.perf_counter() - t0
    N = dims[0] * dims[1] * dims[2]
    omp_threads(os.cpu_count())
    return dict(value=N * n / dt / 1e6, unit=UNIT, cores=cores, kind="oracle",
                sample=f"{n} steps of a {dims[0]}x{dims[1]}x{dims[2]} sub-box of the workload "
                       f"({len(w['particles'])} spheres), FP64 C oracle, OpenMP on {cores} threads",
                seconds=dt)


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    import oracle as O
    from paper_2505_10171_gb300 import workloads as W
    budget = 150.0
    chosen = None
    for dims in ((128, 128, 48), (96, 96, 40), (64, 64, 32), (48, 48, 24)):
        w = W.cfg2_crop(*dims)
        s = O.from_workload(w)
        t0 = time.perf_counter()
        s.step(1)
        t1 = time.perf_counter() - t0
        chosen = (dims, w, s)
        if t1 * (args.steps + args.warmup) <= budget:
            break
    dims, w, s = chosen
    s.step(args.warmup)
    t0 = time.perf_counter()
    s.step(args.steps)
    dt = time.perf_counter() - t0
    N = dims[0] * dims[1] * dims[2]
    value = N * args.steps / dt / 1e6
    cores = os.cpu_count()
    line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=dt / args.steps * 1e3, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=WORKLOAD, sample=f"{dims[0]}x{dims[1]}x{dims[2]} sub-box per step"),
                cpu_baseline=dict(value=value, unit=UNIT, cores=cores, kind="oracle",
                                  sample=f"each step = one FP64 oracle time step of a {dims[0]}x{dims[1]}x{dims[2]} "
                                         f"sub-box of the workload ({len(w['particles'])} spheres)"),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def build_context(lbm, w, precision, stream_handle, store_velocity=0):
    p = dict(w["params"], store_velocity=store_velocity, diag_interval=0)
    ctx = lbm.Context(p, precision, stream=stream_handle)
    if w.get("mask") is not None:
        ctx.lbm_set_solid_mask(w["mask"])
    if w.get("particles"):
        ctx.lbm_add_particles(w["particles"])
    return ctx


def timed_steps(torch, ctx, stream, K, profile):
    """K steps between CUDA events on the context's stream."""
    ctx.lbm_profile(1 if profile else 0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.lbm_step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = ctx.lbm_profile_read() if profile else None
    launches = ctx.lbm_last_launch_count()
    ctx.lbm_profile(0)
    return ms, prof, launches


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=300)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp16", "bf16", "fp64"], default="fp32")
    ap.add_argument("--no-extra", action="store_true", help="skip the 16-bit and batched extra measurements")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline sample")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    # CPU baseline first (no process forked after the GPU is touched)
    cpu = cpu1 = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_sample()
        cpu1 = oracle_sample(budget_s=10.0, threads=1)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2505_10171_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    if dist is not None:
        dist.barrier()
    from paper_2505_10171_gb300 import lbm
    from paper_2505_10171_gb300 import workloads as W

    stream = torch.cuda.Stream()
    w = W.cfg2()
    N = 256 * 128 * 128
    ctx = build_context(lbm, w, args.precision, stream.cuda_stream)
    ctx.lbm_init_fields(w["phi"])
    ctx.lbm_step(args.warmup)
    torch.cuda.synchronize()

    # timed region: K steps replayed from the captured step graph (the
    # production path: particle forces run beside the fluid kernels)
    clocks = ClockSampler(local)
    clocks.start()
    if dist is not None:
        dist.barrier()
    ms, _, launches = timed_steps(torch, ctx, stream, args.steps, profile=False)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    clk = clocks.stop()
    # the same K steps launched one kernel at a time between CUDA events on the
    # launching stream: per-kernel durations for the roofline
    ms_prof, prof, _ = timed_steps(torch, ctx, stream, args.steps, profile=True)
    diag = ctx.lbm_diagnostics()
    ctx.close()

    value = world * N * args.steps / (ms * 1e-3) / 1e6
    peaks = measured_peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6.8 TB/s"
    dom = max(prof, key=lambda k: prof[k]["ms"])
    dom_ms = prof[dom]["ms"] / max(1, prof[dom]["launches"])
    dom_bytes = population_bytes_per_node(dom, args.precision) * N
    dom_design = design_bytes_per_node(dom, args.precision) * N
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9 if dom_bytes else None
    step_bytes = method_bytes_per_lu(args.precision) * N
    design_step = sum(design_bytes_per_node(k, args.precision) for k in ("phi", "grad_wetting", "collide"))
    roofline = dict(bound="hbm", kernel=dom, achieved=achieved, peak=hbm, unit="GB/s",
                    frac=(achieved / hbm) if achieved else None,
                    traffic=ncu_traffic(dom, args.precision), peak_source=peak_src,
                    algorithmic_bytes_per_launch=dom_bytes, avg_launch_ms=dom_ms,
                    design_bytes_per_launch=dom_design,
                    design_frac=dom_design / (dom_ms * 1e-3) / 1e9 / hbm)
    stage_ms = {k: round(v["ms"] / max(1, v["launches"]), 5) for k, v in prof.items() if v["launches"]}
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype=DTYPE[args.precision], data="synthetic",
                config=dict(workload=WORKLOAD, nodes=N, precision=f"{args.precision} offset population storage",
                            parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                            l2="inputs larger than L2 (populations %.0f MB)" % (2 * step_bytes / 2 / 1e6)),
                roofline=roofline,
                step_roofline_frac=(value * 1e6 * step_bytes / N) / (hbm * 1e9),
                bytes_per_lu=dict(method=method_bytes_per_lu(args.precision), moved=design_step,
                                  note="method: read + write of 38 populations; moved: every population and "
                                       "per-node field byte the fluid kernels read or write once"),
                stage_ms_per_launch=stage_ms,
                value_profiled=world * N * args.steps / (ms_prof * 1e-3) / 1e6,
                gpu_launches=launches, clocks=clk, mass=dict(rho_a=diag[0], rho_b=diag[1]))
    if cpu:
        line["cpu_baseline"] = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}
        line["cpu_baseline"]["cpu_model"] = cpu_model()
        if cpu1:
            line["cpu_baseline"]["single_thread"] = {k: cpu1[k] for k in ("value", "unit", "cores", "sample")}

    if rank == 0:
        line["e2e"] = e2e_measure(torch, lbm, W, args, stream)
        if not args.no_extra and world == 1:
            line["extra"] = extra_measure(torch, lbm, W, args, stream, N)
            for prec in ("fp16", "bf16"):
                line["extra"][prec]["speedup_over_fp32_step"] = line["extra"][prec]["value"] / value
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def e2e_measure(torch, lbm, W, args, stream):
    """The same metric through the C ABI with host buffers: pinned-host upload of
    the initial order parameter, K single-step calls, every step's per-particle
    records written into a page-locked host ring by the step itself
    (lbm_set_record_ring, one slot per step), and a final synchronising host
    read of phi, which the timed region includes."""
    import numpy as np
    w = W.cfg2()
    N = 256 * 128 * 128
    nparts = len(w["particles"])
    phi_h = torch.from_numpy(w["phi"]).pin_memory().numpy()
    out_h = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
    K = args.steps
    rec_h = torch.zeros((K, nparts * lbm.PARTICLE_RECORD), dtype=torch.float64).pin_memory().numpy()
    ctx = build_context(lbm, w, args.precision, stream.cuda_stream)
    ctx.lbm_init_fields(phi_h)
    ctx.lbm_set_record_ring(rec_h)  # before the graphs are captured
    ctx.lbm_step(args.warmup)
    for k in range(2):  # both single-step graphs captured before the timed region
        ctx.lbm_step(1)
    torch.cuda.synchronize()
    rec_h[:] = np.nan  # every slot must be written again by the timed steps
    t0 = time.perf_counter()
    ctx.lbm_init_fields(phi_h)
    for k in range(K):
        ctx.lbm_step(1)
    ctx.lbm_read_fields(lbm.FIELD_PHI, out=out_h)
    dt = time.perf_counter() - t0
    if not np.isfinite(rec_h).all():
        raise RuntimeError("particle records missing or non-finite in the end-to-end run")
    ctx.close()
    return dict(value=N * K / dt / 1e6, unit=UNIT, h2d_bytes_per_step=8 * N / K,
                d2h_bytes_per_step=8 * lbm.PARTICLE_RECORD * nparts + 8 * N / K)


def extra_measure(torch, lbm, W, args, stream, N):
    """FP16/BF16 offset storage on the same workload, and the batched sweep."""
    out = {}
    K = max(50, args.steps // 4)
    for prec in ("fp16", "bf16"):
        w = W.cfg2()
        ctx = build_context(lbm, w, prec, stream.cuda_stream)
        ctx.lbm_init_fields(w["phi"])
        ctx.lbm_step(args.warmup)
        ms, prof, _ = timed_steps(torch, ctx, stream, K, profile=True)
        ms_g, _, _ = timed_steps(torch, ctx, stream, K, profile=False)
        ctx.close()
        col = prof["collide"]
        cms = col["ms"] / max(1, col["launches"])
        out[prec] = dict(value=N * K / (ms_g * 1e-3) / 1e6, value_profiled=N * K / (ms * 1e-3) / 1e6,
                         collide_ms=cms, collide_gbs=design_bytes_per_node("collide", prec) * N / (cms * 1e-3) / 1e9,
                         steps=K)
    # the non-tensor arithmetic ceiling of the 16-bit modes (their collision
    # is issue-bound): measured FP32 FMA throughput against the nominal rate
    # (152 SMs x 128 FP32 lanes x 2 FLOP x the maximum SM clock)
    fma = lbm.lbm_fp32_fma_peak()
    nominal = 152 * 128 * 2 * 2.07e9 / 1e12
    out["alu"] = dict(fp32_fma_peak_tflops=fma, unit="TFLOP/s", nominal_tflops=nominal, frac_of_nominal=fma / nominal)
    out["batched"] = batched_measure(torch, lbm, W, args, stream)
    out["stated_error"] = error_measure(lbm, W, stream)
    return out


def batched_measure(torch, lbm, W, args, stream):
    """The 96-instance sweep of uneven domains: one batched FP16 context with
    the autotuned launch shape (graph-captured steps), against the same
    instances stepped one at a time as plain FP32 contexts (the per-instance
    baseline), both timed with CUDA events over the same number of steps after
    warm-up.  Accuracy: the smallest and the largest instance after the same
    steps from the same start, batched FP16 and single FP32 each against a
    single FP64 run (phi, u over common fluid nodes)."""
    import numpy as np

    ws = W.cfg4()
    warm, Kb = 20, max(20, args.steps // 20)
    params = [dict(w["params"], store_velocity=1) for w in ws]

    def one(k, prec):
        c = lbm.Context(params[k], prec, stream=stream.cuda_stream)
        c.lbm_add_particles(ws[k]["particles"])
        c.lbm_init_fields(ws[k]["phi"])
        return c

    ctx = lbm.Context(params, "fp16", stream=stream.cuda_stream)
    nodes = 0
    for k, w in enumerate(ws):
        ctx.lbm_add_particles(w["particles"], inst=k)
        ctx.lbm_init_fields(w["phi"], inst=k)
        nodes += ctx.num_nodes(k)
    tile, zc, _ = ctx.lbm_autotune(4)
    tuned_steps = ctx.lbm_diagnostics()[2]
    ms_b, _, launches = timed_steps(torch, ctx, stream, Kb, profile=False)
    steps_b = ctx.lbm_diagnostics()[2]
    sizes = [ctx.num_nodes(k) for k in range(len(ws))]
    picks = sorted({int(np.argmin(sizes)), int(np.argmax(sizes))})
    got16 = {k: (ctx.fields(k), ctx.owner(k)) for k in picks}
    ctx.close()
    # per-instance plain FP32 runs, one context at a time
    total_ms = 0.0
    for k in range(len(ws)):
        c = one(k, "fp32")
        c.lbm_step(warm)
        ms, _, _ = timed_steps(torch, c, stream, Kb, profile=False)
        total_ms += ms
        c.close()
    acc = {}
    for k in picks:
        ref = one(k, "fp64")
        ref.lbm_step(int(steps_b))
        f0, o0 = ref.fields(), ref.owner()
        ref.close()
        c = one(k, "fp32")
        c.lbm_step(int(steps_b))
        f32, o32 = c.fields(), c.owner()
        c.close()
        f16, o16 = got16[k]

        def rl2(a, b):
            return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

        e = {}
        for name, f, o in (("batched_fp16", f16, o16), ("single_fp32", f32, o32)):
            fl = (o0 == 0) & (o == 0)
            e[name] = dict(phi=rl2(f["phi"][fl], f0["phi"][fl]), u=rl2(f["u"][:, fl], f0["u"][:, fl]))
        acc[f"instance {k} ({sizes[k]} nodes)"] = e
    value = nodes * Kb / (ms_b * 1e-3) / 1e6
    base = nodes * Kb / (total_ms * 1e-3) / 1e6
    return dict(value=value, unit=UNIT, instances=len(ws), nodes=nodes, steps=Kb, launches_per_step=launches / Kb,
                shape=dict(tile=tile, grad_zchunk_per_instance=sorted(set(zc)), autotune_steps=int(tuned_steps)),
                per_instance_fp32=dict(value=base, unit=UNIT, note="96 plain FP32 contexts run one after another, "
                                       "same steps each after %d warm-up steps" % warm),
                speedup_over_per_instance_fp32=value / base,
                error_vs_fp64_after_steps=int(steps_b), accuracy=acc)


def error_measure(lbm, W, stream):
    """rel-L2 of density, order parameter, velocity (fluid nodes on both sides)
    and the stacked per-particle hydrodynamic and capillary forces of each
    storage form against the FP64 path (which the parity tests hold to the
    oracle within 1e-12), after 200 steps of the 48x32x32 drop-sphere case."""
    import numpy as np

    w = W.cfg1()

    def run(prec):
        ctx = lbm.Context(dict(w["params"], store_velocity=1), prec, stream=stream.cuda_stream)
        ctx.lbm_add_particles(w["particles"])
        ctx.lbm_init_fields(w["phi"])
        ctx.lbm_step(w["steps"])
        f, own, parts = ctx.fields(), ctx.owner(), ctx.lbm_particle_forces()
        ctx.close()
        return f, own, np.concatenate([parts[:, 0:3], parts[:, 6:9]])

    def rl2(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    f0, o0, F0 = run("fp64")
    out = dict(reference="fp64 path, 48x32x32 drop + sphere, 200 steps", bar={"fp32": 1e-4, "reduced": 2e-3})
    for prec in ("fp32", "fp16", "bf16"):
        f, o, F = run(prec)
        fl = (o0 == 0) & (o == 0)
        out[prec] = dict(rho=rl2((f["rho_a"] + f["rho_b"])[fl], (f0["rho_a"] + f0["rho_b"])[fl]),
                         phi=rl2(f["phi"][fl], f0["phi"][fl]), u=rl2(f["u"][:, fl], f0["u"][:, fl]),
                         force=float(np.linalg.norm(F - F0) / max(np.linalg.norm(F0), 1e-3 * np.sqrt(F0.size))))
    return out


if __name__ == "__main__":
    main()
