"""Benchmark: velocity DOF-stage updates per second of SSP-RK3 with the hybrid-mixed solve.

One step = one SSP-RK3 time step (three stages; each stage = element residual
and condensation, facet PCG solve, recovery) on the double shear layer,
256 x 256 split squares of [0, 2pi]^2 (131072 triangles), BDM_3, nu = 1e-4.
The timed form is the mixed-precision one: element kernels and the facet PCG in
double-float arithmetic on the FP32 units, the PCG preconditioned by the FP32
Fourier-space inverse of the facet operator. The FP64 form is timed on the
same workload and its state compared with the mixed one.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--mode step|ensemble|adjoint] [--workload NAME]

N > 1 (torchrun, one rank per GPU): in the step mode every rank advances its own
replica of the workload (independent instances, weak scaling); in the ensemble
mode the instances are dealt out to the ranks (strong scaling). Rank 0 prints
the line; times are the maximum over ranks.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "velocity DOF-stage updates/s incl. hybrid-mixed solve; mixed vs FP64 at 1e-9 rel"
UNIT = "velocity DOF-stage updates/s"
WORKLOAD = "shear_n256_k3"
SAMPLE_N = 32          # oracle sample: same workload on a 32 x 32 split-square mesh
L2_FLUSH_BYTES = 512 << 20

# DRAM bytes (read + write) per launch of the dominant kernel on the bench workload, averaged
# over the three stages of a step (the first stage reads one state, the others two), from the
# ncu capture summarised in profiles/; used only while the stage-kernel sources still hash to
# the captured `sha`, else the line reports null.
NCU_TRAFFIC = {"stage_residual": {"sha": "62f71c3ca9c15082", "n_tri": 131072, "bytes": 40963755,
                                  "source": "profiles/k_stage_df2_shear_n256_k3.md"}}


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def reduce_over_ranks(values, op, dist=None, device="cpu"):
    """Element-wise max or sum of a list of floats over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return [float(v) for v in t.tolist()]


def job_rate(local_units, local_seconds, dist=None, device="cpu"):
    """Whole-job throughput: the units processed by all ranks / the slowest rank's time."""
    units, = reduce_over_ranks([local_units], "sum", dist, device)
    secs, = reduce_over_ranks([local_seconds], "max", dist, device)
    return units / secs, units, secs


def shard(n, rank, world):
    """Indices of the independent instances rank `rank` of `world` advances (round robin)."""
    return list(range(rank, n, world))


def dof_stage_units(n_tri, k, steps):
    return n_tri * (k + 1) * (k + 2) * 3 * steps


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """SM clock and clock-event reasons of one GPU during a region. Read-only NVML queries
    (libnvidia-ml through ctypes) polled every 2 ms by a thread, so that a region of a few tens
    of milliseconds still gets samples; `nvidia-smi -lms 200` where NVML cannot be loaded."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits (nvml.h): SW power cap, HW slowdown, SW / HW thermal slowdown
    REASON_BITS = (("sw_power_cap", 0x4), ("hw_slowdown", 0x8), ("sw_thermal_slowdown", 0x20),
                   ("hw_thermal_slowdown", 0x40))

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.thread = None
        self.samples = []
        self.source = None

    def _nvml(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None
        dev = ctypes.c_void_p()
        ok = False
        try:   # the CUDA device by its UUID (NVML may number the GPUs differently from CUDA)
            import torch
            u = str(torch.cuda.get_device_properties(self.index).uuid)
            u = u if u.startswith("GPU-") else "GPU-" + u
            ok = lib.nvmlDeviceGetHandleByUUID(ctypes.c_char_p(u.encode()), ctypes.byref(dev)) == 0
        except Exception:
            ok = False
        if not ok and lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(dev)) != 0:
            lib.nvmlShutdown()
            return None
        reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        return lib, dev, reasons_fn

    def __enter__(self):
        import ctypes
        import threading
        self.samples = []
        try:
            handles = self._nvml()
        except (OSError, AttributeError):
            handles = None
        if handles is not None:
            lib, dev, reasons_fn = handles
            self.source = "nvml"
            self.stop = threading.Event()

            def poll():
                clk, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
                while not self.stop.is_set():
                    if (lib.nvmlDeviceGetClockInfo(dev, 1, ctypes.byref(clk)) == 0 and       # NVML_CLOCK_SM
                            lib.nvmlDeviceGetMaxClockInfo(dev, 1, ctypes.byref(mx)) == 0 and
                            reasons_fn(dev, ctypes.byref(rs)) == 0):
                        self.samples.append((float(clk.value), float(mx.value), int(rs.value)))
                    self.stop.wait(0.002)
                lib.nvmlShutdown()

            self.thread = threading.Thread(target=poll, daemon=True)
            self.thread.start()
            return self
        self.source = "nvidia-smi"
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.thread is not None:
            self.stop.set()
            self.thread.join(timeout=5)
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        if self.source == "nvml":
            for c, m, r in self.samples:
                sm.append(c)
                smax.append(m)
                for n, bit in self.REASON_BITS:
                    if r & bit:
                        reasons.add(n)
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in getattr(self, "lines", []):
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0,
                    "source": self.source}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "min_sm_mhz": min(sm), "source": self.source}


def element_kernel_sha():
    h = hashlib.sha256()
    for n in ("k_stage_df.cu", "ktables.cuh", "dfloat.cuh", "kcommon.cuh", "device.cuh"):
        with open(os.path.join(ROOT, "paper_1808_04669_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def stage_flops_per_triangle(k, tabulated=True):
    """Flops of the stage kernel per triangle (FMA = 2), counted from its loops: the volume rule
    has 3, 7, 16 points for k = 1, 2, 3 (fully symmetric, degree 3k - 1). With
    `tabulated` (meshes of at most 4 geometry classes, mixed form) the facet normal derivatives
    of the basis come from per-class tables: two sums per trace and per test instead of three."""
    ns = (k + 1) * (k + 2) // 2
    nd = 2 * ns
    nq = {1: 3, 2: 7, 3: 16}[k]
    nqf = (3 * k + 2) // 2
    vol = nq * (2 * (6 * ns + 4 * ns) + 40)              # trace/gradient sums, flux, test sums
    per_pt = (8 * ns + 4 * ns) if tabulated else (12 * ns + 6 * ns)
    fac = 3 * nqf * (2 * per_pt + 30)                      # both traces, flux, test sums
    out = 3 * nd + 2 * nd * nd + 2 * 3 * (k + 1) * nd    # stage combination, P f, G f
    return vol + fac + out


def lattice_solver_bytes(n_facet, k, iters, solves):
    """Algorithmic DRAM bytes of the mixed-form lattice (Fourier-preconditioned) facet solves.

    Vectors are double-float (8 B per DOF), z is FP32 (4 B); the spectrum holds half the
    wavenumbers (4 B per DOF per pass) and the FP32 deflated eigen form of the symbol
    (C + 1 + C(C+1)/2 complex entries per wavenumber: 4 (C + 1 + C(C+1)/2) / C B per DOF),
    C = 3(k+1). Per DOF and CG iteration: SpMV pass 36 B (read z, p, q; write p, q); update +
    forward rows 52 B (read r, q, lam, p; write r, lam, spectrum); columns 8 B + symbol; inverse
    rows 20 B (read spectrum, r, z_old; write z); plus 20 B of stencil ids per facet. Per solve:
    g assembly with the warm-start history (read two entries, shift one), the first residual and
    one more preconditioner application, 124 B + symbol per DOF; the new multipliers are copied
    into the history, 16 B per DOF.
    """
    nl = n_facet * (k + 1)
    C = 3 * (k + 1)
    sym = 4 * (C + 1 + C * (C + 1) // 2) / C
    per_iter = nl * (36 + 52 + 8 + sym + 20) + 20 * n_facet
    per_solve = nl * (124 + 16 + sym) + 20 * n_facet
    return iters * per_iter + solves * per_solve


def solver_bytes(n_facet, k, iters, sweeps, solves):
    """Algorithmic DRAM bytes of the block-Jacobi mixed facet solves.

    Per inner FP32 CG iteration: 11 vector passes of 4 B per multiplier DOF
    (read z, p_old; write p_new, q; read x, p_new, r, q; write x, r, z) plus
    24 B of stencil indices per facet. Per FP64 refinement sweep: read lam and
    g (8 B each), write the FP32 residual (4 B), then lam += d (8 + 4 + 8 B)
    per DOF, plus 20 B of indices per facet. Per solve: assemble g from the two
    element sides (2 x 4 B per DOF read, 8 B write) and rescale lam (16 B).
    """
    nl = n_facet * (k + 1)
    per_iter = 11 * 4 * nl + 24 * n_facet
    per_sweep = 40 * nl + 20 * n_facet
    per_solve = 32 * nl + 9 * n_facet
    return iters * per_iter + sweeps * per_sweep + solves * per_solve


def stage_bytes_per_triangle(k):
    """Algorithmic DRAM bytes of one stage-kernel launch per triangle (8 B per value: FP64, or a
    double-float pair): read the states u^n and u' (one state in the first SSP-RK3 stage, where
    both are u^n: 5/3 states on average), write h = P f (n_u values) and G f (3 (k+1) values).
    Neighbour traces are re-read from L2."""
    nd = (k + 1) * (k + 2)
    return 8 * (5.0 / 3.0 * nd + nd + 3 * (k + 1))


def sm_count():
    """Streaming multiprocessors of the current device."""
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def fp64_peak_tflops(sm_mhz, sms):
    """FP64 ALU peak: 2 FP64 FMA per clock per SM (an FMA-chain probe measured 1.20 TFLOP/s) x SMs."""
    return 2 * 2 * sms * sm_mhz * 1e6 / 1e12


DF_OPS_PER_FMA = 12


def dfl_peak_tflops(sm_mhz, sms):
    """Double-float ALU peak in algorithmic flops (modelled): 128 FP32 lanes per SM x SMs x clock,
    divided by the 12 FP32 operations of one double-float multiply-add (exact product 2, cross
    terms 2, TwoSum 6, error accumulation 2), times 2 flops per multiply-add."""
    return 128 * sms * sm_mhz * 1e6 / DF_OPS_PER_FMA * 2 / 1e12


def workload_label(w, N, n_tri):
    ic = {"shear": "double shear layer", "tgv": "Taylor-Green", "spectrum": "random-spectrum field (seed %d)" % w.seed}
    dom = "[0,2pi]^2" if w.L > 1.5 else "unit square"
    return "%s, %s periodic, %dx%d split squares (%d triangles), BDM_%d, nu=%g, SSP-RK3, CFL dt" % (
        ic.get(w.ic, w.ic), dom, N, N, n_tri, w.k, w.nu)


def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1808_04669_gb300 import build as _b
    _b.build()
    import paper_1808_04669_gb300 as g
    import synth
    workload = args.workload or WORKLOAD
    vid, X, vals, dt = synth.make_workload(workload, N=args.n)
    w = synth.WORKLOADS[workload]
    k = w.k
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_steps(mesh, K, W, profile=False):
        for _ in range(W):
            mesh.rk3_step(dt, 1)
        torch.cuda.synchronize()
        if profile:
            mesh.profile(2)
            mesh.profile(1)
        st0 = mesh.solver_stats()
        total = 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(K):
            flush.fill_(1.0)                       # evict L2 between timed steps (not timed)
            barrier()
            e0.record(stream)
            mesh.rk3_step(dt, 1)
            e1.record(stream)
            barrier()
            total += e0.elapsed_time(e1)
        prof = mesh.profile(0) if profile else None
        st1 = mesh.solver_stats()
        return total, prof, st0, st1

    mixed = g.DGMesh(vid, X, k, w.nu, precision=g.MIXED, stream=stream.cuda_stream)
    mixed.set_velocity(vals)
    mixed.project_divfree()
    u0 = mixed.get_velocity()
    sampler = ClockSampler(local)
    with sampler:
        t_ms, prof, st0, st1 = timed_steps(mixed, args.steps, args.warmup, profile=True)
    clocks = sampler.summary()
    value, units, t_s = job_rate(dof_stage_units(mixed.n_tri, k, args.steps), t_ms * 1e-3, dist, "cuda")
    t_ms = t_s * 1e3
    u_mixed = mixed.get_velocity()

    # the same steps with the tensor-core (tcgen05) recovery, a secondary measurement
    tc_line = None
    try:
        tcm = g.DGMesh(vid, X, k, w.nu, precision=g.MIXED, stream=stream.cuda_stream)
        tcm.set_tensor_cores(1)
        tcm.set_velocity(u0)
        t_tc, prof_tc, _, _ = timed_steps(tcm, args.steps, args.warmup, profile=True)
        rel_tc = float(np.linalg.norm(tcm.get_velocity() - u_mixed) / np.linalg.norm(u_mixed))
        rec = prof_tc.get("recover", (0.0, 1))
        tc_line = {"ms_per_step": t_tc / args.steps, "recover_ms_per_launch": rec[0] / max(rec[1], 1),
                   "kernel_ms": {k_: v[0] for k_, v in prof_tc.items() if v[1]},
                   "vs_double_float_recovery_rel_l2": rel_tc,
                   "kernel": "k_recover_tc<%d>: u = [P, -G^T][f; lam] per 128-triangle class tile on tcgen05, "
                             "7 bf16 digit slices per operand, exact FP32 accumulation in TMEM" % k}
        tcm.close()
    except g.DGError as e:
        tc_line = {"unavailable": str(e)}

    # FP64 form on the same initial state and step count
    fp64 = g.DGMesh(vid, X, k, w.nu, precision=g.FP64, stream=stream.cuda_stream)
    fp64.set_velocity(u0)
    t64, prof64, s640, s641 = timed_steps(fp64, args.steps, args.warmup, profile=True)
    u64 = fp64.get_velocity()
    rel = float(np.linalg.norm(u_mixed - u64) / np.linalg.norm(u64))
    value64, _, t64_s = job_rate(dof_stage_units(fp64.n_tri, k, args.steps), t64 * 1e-3, dist, "cuda")
    t64 = t64_s * 1e3
    diag = mixed.diagnostics()

    # end to end through the public API with host buffers: per step, copy the state in from
    # pinned host memory, advance one step, copy the state back
    host = torch.from_numpy(u_mixed.copy()).pin_memory()
    e2e_mesh = g.DGMesh(vid, X, k, w.nu, precision=g.MIXED, stream=stream.cuda_stream)
    e2e_mesh.set_velocity(host)
    for _ in range(args.warmup):
        e2e_mesh.rk3_step(dt, 1)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_mesh.set_velocity(host)
        e2e_mesh.rk3_step(dt, 1)
        e2e_mesh.get_velocity(host)
    barrier()
    value_e2e, _, _ = job_rate(dof_stage_units(mixed.n_tri, k, args.steps), time.perf_counter() - t0, dist, "cuda")
    lat_bytes = host.numel() * 8

    # roofline of the dominant kernel in the timed region
    name = max(prof, key=lambda n_: prof[n_][0])
    ms_k, n_k = prof[name]
    per_launch_s = ms_k * 1e-3 / max(n_k, 1)
    iters = st1["total_iters"] - st0["total_iters"]
    sweeps = st1["total_sweeps"] - st0["total_sweeps"]
    solves = st1["solves"] - st0["solves"]
    peaks = measured_peaks()
    traffic = None
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    sms = sm_count()
    hbm_peak = peaks.get("hbm_gbs")

    def hbm_part(nbytes):
        gbs = nbytes / per_launch_s / 1e9
        return {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": (gbs / hbm_peak) if hbm_peak else None,
                "bytes_per_launch": nbytes, "peak_source": "MEASURED_PEAKS.json hbm_gbs"}

    if name.startswith("stage_residual"):
        flops = stage_flops_per_triangle(k, tabulated=mixed.n_class <= 4) * mixed.n_tri
        achieved = flops / per_launch_s / 1e12
        peak = dfl_peak_tflops(sm_mhz, sms)
        tr = NCU_TRAFFIC.get("stage_residual")
        if tr and tr.get("sha") == element_kernel_sha() and tr.get("n_tri") == mixed.n_tri:
            traffic = tr["bytes"]
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic,
                "kernel": "%s<%d> (stage residual + condensation, double-float on the FP32 pipes)"
                          % ("k_stage_df2" if mixed.n_class <= 4 else "k_stage_df", k),
                "peak_source": "modelled: 128 FP32 lanes/SM x %d SMs x median SM clock %.0f MHz / %d FP32 ops "
                               "per double-float multiply-add x 2 flops" % (sms, sm_mhz, DF_OPS_PER_FMA),
                "hbm": hbm_part(stage_bytes_per_triangle(k) * mixed.n_tri)}
    else:
        if name.startswith("facet_pcg_fft"):
            nbytes = lattice_solver_bytes(mixed.n_facet, k, iters, solves)
        else:
            nbytes = solver_bytes(mixed.n_facet, k, iters, sweeps, solves)
        achieved = nbytes / max(n_k, 1) / per_launch_s / 1e9
        peak = peaks.get("hbm_gbs")
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if peak else None, "traffic": traffic, "kernel": name,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
    launches = sum(v[1] for v in prof.values())
    total_prof_ms = sum(v[0] for v in prof.values())
    # FP64 form: its dominant kernel is the FP64 stage kernel, bound by the FP64 pipe; the HBM
    # fraction of the same launches is reported beside it
    name64 = max(prof64, key=lambda n_: prof64[n_][0])
    ms64, n64 = prof64[name64]
    per64_s = ms64 * 1e-3 / max(n64, 1)
    roof64 = {"kernel": name64, "ms_per_launch": per64_s * 1e3,
              "share_of_device_time": ms64 / sum(v[0] for v in prof64.values())}
    if name64.startswith("stage_residual"):
        a64 = stage_flops_per_triangle(k, tabulated=False) * fp64.n_tri / per64_s / 1e12
        p64 = fp64_peak_tflops(sm_mhz, sms)
        b64 = stage_bytes_per_triangle(k) * fp64.n_tri
        roof64.update({"bound": "alu", "achieved": a64, "peak": p64, "unit": "TFLOP/s", "frac": a64 / p64,
                       "peak_source": "derived: 2 FP64 FMA/clock/SM x %d SMs x median SM clock %.0f MHz x 2 flops"
                                      % (sms, sm_mhz),
                       "hbm": {"achieved": b64 / per64_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                               "frac": (b64 / per64_s / 1e9 / hbm_peak) if hbm_peak else None,
                               "bytes_per_launch": b64, "peak_source": "MEASURED_PEAKS.json hbm_gbs"}})

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32x2 (double-float) element kernels and PCG vectors, f32 Fourier preconditioner, f64 state",
        "data": "synthetic (double shear layer sampled at lattice points, seeded)",
        "config": {"workload": workload_label(w, args.n or w.N, mixed.n_tri),
                   "N": args.n or w.N, "k": k, "nu": w.nu, "dt": dt,
                   "n_tri": mixed.n_tri, "n_facet": mixed.n_facet, "broken_velocity_dofs": mixed.n_vel_dofs,
                   "multiplier_dofs": mixed.n_lam_dofs, "l2": "flushed between timed steps (512 MiB write)",
                   "parallelism": "replicas (one independent instance per GPU)"},
        "clocks": clocks,
        "e2e": {"value": value_e2e, "unit": UNIT,
                "h2d_bytes_per_step": lat_bytes, "d2h_bytes_per_step": lat_bytes},
        "gpu_launches": launches,
        "roofline": roof,
        "fp64": {"value": value64, "ms_per_step": t64 / args.steps, "cg_iters_per_solve":
                 (s641["total_iters"] - s640["total_iters"]) / max(s641["solves"] - s640["solves"], 1),
                 "roofline": roof64},
        "mixed_vs_fp64_rel_l2": rel,
        "tensor_core_recovery": tc_line,
        "solver": {"iters_per_solve": iters / max(solves, 1), "sweeps_per_solve": sweeps / max(solves, 1),
                   "preconditioner": mixed.solver_stats()["preconditioner"],
                   "dominant_kernel_ms_per_launch": per_launch_s * 1e3,
                   "kernel_ms": {k_: v[0] for k_, v in prof.items() if v[1]},
                   "share_of_device_time": {k_: v[0] / total_prof_ms for k_, v in prof.items() if v[1]}},
        "diagnostics": {"energy": diag["energy"], "max_div": diag["max_div"], "max_jump": diag["max_jump"]},
    }
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(1)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


def run_ensemble(args):
    """Ensemble workload: 64 instances on the unit square, N ~ U{32..256}, k ~ U{1,2,3},
    log10 nu ~ U[-5,-2], Taylor-Green or random-spectrum initial data (seeds 100+i), mixed
    precision, advanced together by dg_batch_rk3_step (one captured CUDA graph per step)."""
    import numpy as np
    import torch
    from paper_1808_04669_gb300 import build as _b
    _b.build()
    import paper_1808_04669_gb300 as g
    import synth
    rank, world, local = env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    rng = np.random.Generator(np.random.PCG64(1))
    n_inst = args.instances
    mine = set(shard(n_inst, rank, world))
    meshes, dts, units_per_step = [], [], 0
    for i in range(n_inst):
        N = int(rng.integers(32, 257))
        k = int(rng.integers(1, 4))
        nu = float(10.0 ** rng.uniform(-5, -2))
        tgv = rng.uniform() < 0.5
        if i not in mine:
            continue
        vid, X = synth.split_square_mesh(N, L=1.0)
        f = synth.taylor_green(1.0) if tgv else synth.random_spectrum_velocity(100 + i, L=1.0)
        vals = synth.sample_lattice(f, X, k, grid=None if (tgv or k * N <= 64) else (k * N, 1.0))
        dts.append(synth.cfl_dt(X, k, float(np.sqrt((vals ** 2).sum(-1)).max()), nu))
        m = g.DGMesh(vid, X, k, nu, precision=g.MIXED)
        m.set_velocity(vals)
        m.project_divfree()
        meshes.append(m)
        units_per_step += dof_stage_units(m.n_tri, k, 1)
    batch = g.DGBatch(meshes)
    batch.set_lanes(args.lanes)
    dts = np.array(dts)
    # warm-up: the eager steps that fill every member's multiplier history, then the lane
    # tuner's replays (two per candidate), before the timed region
    batch.rk3_step(dts, max(args.warmup, 14))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch.rk3_step(dts, args.steps)
    torch.cuda.synchronize()
    value, _, t = job_rate(units_per_step * args.steps, time.perf_counter() - t0, dist, "cuda")
    lat, tris = reduce_over_ranks([sum(int(m.solver_stats()["lattice"]) for m in meshes),
                                   sum(m.n_tri for m in meshes)], "sum", dist, "cuda")
    lanes, tune = batch.tuning()
    batch.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    print(json.dumps({"mode": "ensemble", "metric": UNIT + " (ensemble, all instances)",
                      "value": value, "unit": UNIT, "n_gpus": world, "scaling": "strong", "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "instances": n_inst,
                      "triangles": int(tris), "lattice_instances": int(lat),
                      "dtype": "f32x2 (double-float) element kernels and PCG vectors, f32 Fourier preconditioner, f64 state",
                      "config": {"workload": "ensemble of %d periodic unit-square meshes, N~U{32..256}, "
                                             "k~U{1,2,3}, log10 nu~U[-5,-2], seed 1" % n_inst,
                                 "graph": "one captured CUDA graph per step (dg_batch_rk3_step), members on "
                                          "%d parallel branches" % lanes},
                      "lanes": lanes, "lane_tuning_ms_per_step": {str(k_): v for k_, v in tune.items()}}), flush=True)


def run_schemes(args):
    """The other explicit schemes and boundaries (mixed form, device-timed, L2 flushed between
    steps): SSP-RK3, forward Euler and RK4 on the bench workload; SSP-RK3 on the Taylor-Green
    cell in a box with free-slip walls and on a channel with inflow and outflow (multilevel facet
    solves). Units: broken velocity DOFs times the stages of each step."""
    import numpy as np
    import torch
    torch.cuda.set_device(env_rank()[2])
    from paper_1808_04669_gb300 import build as _b
    _b.build()
    import paper_1808_04669_gb300 as g
    import synth
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def timed(mesh, dt, scheme, K, W):
        mesh.step(dt, W, scheme=scheme)
        torch.cuda.synchronize()
        st0 = mesh.solver_stats()
        total = 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(K):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0.record(stream)
            mesh.step(dt, 1, scheme=scheme)
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        st1 = mesh.solver_stats()
        its = (st1["total_iters"] - st0["total_iters"]) / max(st1["solves"] - st0["solves"], 1)
        return total / K, its

    out = {"mode": "schemes", "unit": UNIT, "dtype": "f32x2 (double-float) element kernels, f64 state",
           "data": "synthetic", "steps": args.steps, "warmup": args.warmup, "results": []}
    vid, X, vals, dt = synth.make_workload(WORKLOAD, N=args.n)
    w = synth.WORKLOADS[WORKLOAD]
    for name, scheme, stages in (("ssprk3", g.SSPRK3, 3), ("euler", g.EULER, 1), ("rk4", g.RK4, 4)):
        m = g.DGMesh(vid, X, w.k, w.nu, precision=g.MIXED, stream=stream.cuda_stream)
        m.set_velocity(vals)
        m.project_divfree()
        ms, its = timed(m, dt, scheme, args.steps, args.warmup)
        out["results"].append({"workload": workload_label(w, args.n or w.N, m.n_tri), "scheme": name,
                               "ms_per_step": ms, "iters_per_solve": its,
                               "value": m.n_tri * (w.k + 1) * (w.k + 2) * stages / (ms * 1e-3)})
        m.close()
    N, k, nu = args.n or 128, 3, 1e-4
    vid, X = synth.split_square_mesh(N, L=1.0, periodic=False)
    vals = synth.sample_lattice(synth.taylor_green(L=2.0), X, k)
    dt = synth.cfl_dt(X, k, float(np.abs(vals).max()), nu)
    m = g.DGMesh(vid, X, k, nu, precision=g.MIXED, stream=stream.cuda_stream)
    m.set_velocity(vals)
    m.project_divfree()
    ms, its = timed(m, dt, g.SSPRK3, args.steps, args.warmup)
    out["results"].append({"workload": "Taylor-Green cell, unit square with free-slip walls, %dx%d split squares "
                                       "(%d triangles), BDM_%d, nu=%g, %s PCG" % (N, N, m.n_tri, k, nu,
                                                                                 m.solver_stats()["preconditioner"]),
                           "scheme": "ssprk3", "ms_per_step": ms, "iters_per_solve": its,
                           "value": dof_stage_units(m.n_tri, k, 1) / (ms * 1e-3)})
    m.close()
    # inflow/outflow (Sec. 2.5): a channel [0, 2] x [0, 1] periodic in y, inflow on x = 0 with
    # u_in = (1 + 0.3 sin 2 pi y, 0.2 cos 2 pi y), open outflow on x = 2
    Ny = (args.n or 128) // 2 or 1
    Nx = 2 * Ny
    vid, X = synth.channel_mesh(Nx, Ny, 2.0, 1.0, periodic_y=True)
    kinds = synth.boundary_kinds_by_x(X, 0.0, 2.0)

    def profile(x, y):
        return 1.0 + 0.3 * np.sin(2 * np.pi * y) + 0 * x, 0.2 * np.cos(2 * np.pi * y) + 0 * x
    vals = synth.sample_lattice(profile, X, k)
    dt = synth.cfl_dt(X, k, float(np.sqrt((vals ** 2).sum(-1)).max()), nu)
    m = g.DGMesh(vid, X, k, nu, precision=g.MIXED, stream=stream.cuda_stream, boundary=kinds,
                 inflow=synth.sample_edges(profile, X, k))
    m.set_velocity(vals)
    m.project_divfree()
    ms, its = timed(m, dt, g.SSPRK3, args.steps, args.warmup)
    out["results"].append({"workload": "channel [0,2]x[0,1] periodic in y, inflow x=0, outflow x=2, %dx%d split "
                                       "squares (%d triangles), BDM_%d, nu=%g, %s PCG" % (Nx, Ny, m.n_tri, k, nu,
                                                                                     m.solver_stats()["preconditioner"]),
                           "scheme": "ssprk3", "ms_per_step": ms, "iters_per_solve": its,
                           "value": dof_stage_units(m.n_tri, k, 1) / (ms * 1e-3)})
    m.close()
    out["results"].append(run_three_d(args, g, stream, flush))
    print(json.dumps(out), flush=True)


def run_three_d(args, g, stream, flush):
    """The three-dimensional line (row f2): SSP-RK3 steps of the ABC flow on the periodic cube,
    device-timed with L2 flushed between steps, and the residual kernel alone."""
    import numpy as np
    import torch
    # three dimensions (closed tetrahedral meshes, FP64): the ABC flow on the periodic cube
    # [0, 2 pi]^3 cut into Kuhn tetrahedra, BDM_2, multilevel PCG
    from synth.mesh3 import abc_flow, kuhn_cube_mesh, sample_lattice3
    N3, k3, nu3 = max(2, (args.n or 128) // 8), 2, 1e-3
    vid, X = kuhn_cube_mesh(N3)
    vals = sample_lattice3(abc_flow(), X, k3)
    h3 = 2 * np.pi / N3
    vmax = float(np.sqrt((vals ** 2).sum(-1)).max())
    dt = min(0.1 * h3 / (k3 * k3 * vmax), 0.05 * h3 * h3 / (k3 ** 4 * nu3))
    m3 = g.DGMesh3(vid, X, k3, nu3, stream=stream.cuda_stream)
    m3.set_velocity(vals)
    m3.project_divfree()
    m3.rk3_step(dt, args.warmup)
    torch.cuda.synchronize()
    d0 = m3.diagnostics()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0.record(stream)
        m3.rk3_step(dt, 1)
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    ms = total / args.steps
    d1 = m3.diagnostics()
    its = (d1["total_iters"] - d0["total_iters"]) / max(d1["solves"] - d0["solves"], 1)
    # the stage kernel alone (MODE_RESIDUAL through dg3_eval_residual, lattice output included)
    rbuf = torch.empty((m3.n_tet, m3.n_lat, 3), dtype=torch.float64, device="cuda")
    m3.eval_residual(rbuf)
    torch.cuda.synchronize()
    rt = []
    for _ in range(5):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0.record(stream)
        m3.eval_residual(rbuf)
        e1.record(stream)
        torch.cuda.synchronize()
        rt.append(e0.elapsed_time(e1))
    rms = float(np.median(rt))
    flops = stage3_flops_per_tet(k3) * m3.n_tet
    nd3 = 3 * (k3 + 1) * (k3 + 2) * (k3 + 3) // 6
    sm_mhz, sms = 2070.0, sm_count()
    peak64 = 2 * sms * sm_mhz * 1e6 * 2 / 1e12
    res = {"workload": "ABC flow, periodic cube [0,2pi]^3, %d^3 cubes x 6 Kuhn tetrahedra (%d), BDM_%d, "
                       "nu=%g, FP64, multilevel PCG" % (N3, m3.n_tet, k3, nu3),
           "scheme": "ssprk3", "ms_per_step": ms, "iters_per_solve": its,
           "value": m3.n_tet * nd3 * 3 / (ms * 1e-3),
           "residual_kernel_ms": rms,
           "residual_kernel_fp64_tflops": flops / (rms * 1e-3) / 1e12,
           "fp64_peak_tflops": peak64,
           "peak_source": "derived: 2 FP64 FMA/clock/SM x %d SMs x 2070 MHz x 2 flops" % sms}
    m3.close()
    return res


def stage3_flops_per_tet(k):
    """Flops of the 3-D residual per tetrahedron (FMA = 2), counted from its loops: volume points
    (3k+1)//2 cubed, each evaluating u and grad u (12 ns) and testing (9 ns) plus the flux (~40);
    four faces of ((3k+2)//2)^2 points, each evaluating both traces and normal derivatives (18 ns)
    and testing (9 ns) plus ~30."""
    ns = (k + 1) * (k + 2) * (k + 3) // 6
    nq = ((3 * k + 1) // 2) ** 3
    nqf = ((3 * k + 2) // 2) ** 2
    fma = nq * (21 * ns + 40) + 4 * nqf * (27 * ns + 30)
    return 2 * fma


def run_adjoint(args):
    """Gradient workload: 128 x 128 unit square, BDM_2, nu = 1e-3, random-spectrum u0 (seed 3) and
    target (seed 4), loss 1/2 ||u_K - u*||^2, K = 200 SSP-RK3 steps, checkpoints every 20 steps;
    one timed gradient = dg_rk3_vjp (forward, segment recomputation, reverse sweep)."""
    import numpy as np
    import torch
    from paper_1808_04669_gb300 import build as _b
    _b.build()
    import paper_1808_04669_gb300 as g
    import synth
    w = synth.WORKLOADS["adjoint_n128_k2"]
    vid, X, vals, dt = synth.make_workload(w)
    mesh = g.DGMesh(vid, X, w.k, w.nu)
    tgt = synth.sample_lattice(synth.random_spectrum_velocity(4, L=1.0), X, w.k, grid=(w.k * w.N, 1.0))
    mesh.set_velocity(tgt)
    target = mesh.get_coefficients()
    mesh.set_velocity(vals)
    mesh.project_divfree()
    u0 = mesh.get_coefficients()
    K = args.steps_adjoint
    times = []
    for rep in range(1 + args.reps):
        mesh.set_coefficients(u0)
        mesh.rk3_step(dt, K)
        ubar = mesh.get_coefficients() - target
        mesh.set_coefficients(u0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u0bar, nubar = mesh.rk3_vjp(dt, K, ubar, checkpoint_every=20)
        torch.cuda.synchronize()
        if rep > 0:
            times.append(time.perf_counter() - t0)
    t = min(times)
    print(json.dumps({"mode": "adjoint", "metric": "gradients/s of a %d-step rollout (u0 and nu)" % K,
                      "value": 1.0 / t, "unit": "gradients/s", "seconds_per_gradient": t,
                      "forward_dof_stage_per_s": dof_stage_units(mesh.n_tri, w.k, K) / t,
                      "nubar": nubar, "u0bar_norm": float(np.linalg.norm(u0bar)),
                      "config": {"workload": "128x128 unit square, BDM_2, nu=1e-3, %d steps, checkpoint every 20" % K}}),
          flush=True)


def _oracle_sample_steps(nsteps, warmup=0):
    """Oracle run on the bounded sample; returns (seconds per step, n_tri, k)."""
    import synth
    from oracle import Discretization
    vid, X, vals, dt = synth.make_workload(WORKLOAD, N=SAMPLE_N)
    w = synth.WORKLOADS[WORKLOAD]
    d = Discretization(vid, X, w.k, w.nu)
    d.prepare()                                  # prefactorisation, excluded like the GPU set-up
    U = d.project(d.from_lattice(vals))
    for _ in range(warmup):
        U = d.rk3_step(U, dt, 1)
    times = []
    for _ in range(nsteps):
        t0 = time.perf_counter()
        U = d.rk3_step(U, dt, 1)
        times.append(time.perf_counter() - t0)
    return times, d.n_tri, w.k


def cpu_baseline(nsteps):
    times, n_tri, k = _oracle_sample_steps(nsteps)
    t = sum(times)
    return {"value": dof_stage_units(n_tri, k, nsteps) / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d SSP-RK3 step(s) of the same workload on a %dx%d split-square mesh (%d triangles, BDM_%d), "
                      "after the one-time sparse LU factorisation; NumPy/SciPy single-threaded (OMP/BLAS 1 thread) "
                      "on %d host cores" % (nsteps, SAMPLE_N, SAMPLE_N, n_tri, k, os.cpu_count() or 0)}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    times, n_tri, k = _oracle_sample_steps(args.steps, args.warmup)
    t = sum(times)
    v = dof_stage_units(n_tri, k, args.steps) / t
    cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "each step: one SSP-RK3 step of the same workload on a %dx%d split-square mesh (%d triangles, "
                     "BDM_%d), FP64 NumPy/SciPy oracle, single-threaded" % (SAMPLE_N, SAMPLE_N, n_tri, k)}
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": {"workload": "double shear layer, BDM_3, nu=1e-4; sample "
                                                                   "%dx%d split squares" % (SAMPLE_N, SAMPLE_N)},
                      "cpu_baseline": cpu,
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


def summarize_launches(path):
    """Per-kernel launches, total time and share from an ncu launch-list CSV (gpu__time_duration.sum)."""
    import collections
    import csv
    scale = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0, "s": 1e3,
             "second": 1e3}
    rows = list(csv.reader(open(path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[hi]
    ki, mi, vi, ui = (hdr.index(c) for c in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    agg = collections.OrderedDict()
    for r in rows[hi + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        name = r[ki].split("(")[0].replace("void ", "")
        a = agg.setdefault(name, [0, 0.0])
        a[0] += 1
        a[1] += float(r[vi].replace(",", "")) * scale[r[ui]]
    tot = sum(v[1] for v in agg.values())
    print("%-56s %8s %12s %7s" % ("kernel", "launches", "total ms", "share"))
    for n, (c, t) in sorted(agg.items(), key=lambda x: -x[1][1]):
        print("%-56s %8d %12.3f %6.2f%%" % (n[:56], c, t, 100 * t / tot))
    print("%-56s %8d %12.3f" % ("total", sum(v[0] for v in agg.values()), tot))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", choices=("step", "ensemble", "adjoint", "schemes", "threed"), default="step",
                    help="step: the bench line; ensemble / adjoint / schemes: the batching, gradient, "
                         "time-scheme, boundary and 3-D workloads; threed: the 3-D line alone")
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--lanes", type=int, default=0, help="ensemble: parallel graph branches (0: autotune)")
    ap.add_argument("--steps-adjoint", type=int, default=200)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--summarize-launches", metavar="CSV", help="print a per-kernel summary of an ncu launch list")
    ap.add_argument("--workload", default=None, help="named workload (default %s); the bench line is on the default" % WORKLOAD)
    ap.add_argument("--n", type=int, default=None,
                    help="mesh size override (smaller cases for profiling only; not a bench line)")
    args = ap.parse_args()
    if args.summarize_launches:
        summarize_launches(args.summarize_launches)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "ensemble":
        run_ensemble(args)
    elif args.mode == "adjoint":
        run_adjoint(args)
    elif args.mode == "threed":
        import torch
        torch.cuda.set_device(env_rank()[2])
        from paper_1808_04669_gb300 import build as _b
        _b.build()
        import paper_1808_04669_gb300 as g
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        print(json.dumps({"mode": "threed", "unit": UNIT, "data": "synthetic", "steps": args.steps,
                          "warmup": args.warmup,
                          "results": [run_three_d(args, g, torch.cuda.current_stream(), flush)]}), flush=True)
    elif args.mode == "schemes":
        run_schemes(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(v, "1")
    main()
