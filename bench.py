#!/usr/bin/env python3
"""Benchmark of the KNP-EMI time step (membrane update + assembly + AMG-preconditioned FGMRES).

Workload: the 3D Hodgkin-Huxley scenario on the 64^3 Kuhn mesh of a 100 um cube with one
box cell [0.3, 0.7]^3 (1,114,732 unknowns), stimulus 40 S/m^2 on facets with x < 40 um for
t < 1 ms, dt = 0.05 ms, FGMRES(30) rtol 1e-10, FP64 hierarchy. One "step" is one IMEX time
step; the metric is unknowns x time steps per second. AMG setup (once per run, on P_0) and
topology are excluded, as the paper's "initialization" is; they are reported separately.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs an independent replica (the path does not shard on
this single-GPU pool); value = unknowns x steps of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF*timesteps/s (assembly+AMG-GMRES)"
UNIT = "DOF*steps/s"
WORKLOAD = "3D HH, 64^3 Kuhn tets, 100 um cube, cell [0.3,0.7]^3, 1,114,732 DOF, dt 0.05 ms, rtol 1e-10"
PROFILE_FILE = os.path.join(ROOT, "profiles", "roofline_counters.json")
SAMPLE_NX = 24   # oracle sample: the same scenario on the 24^3 version of its mesh


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--no-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4, 5, 6, 7, 8],
                    help="workload: 2 (default, the headline), 1 (2D leak), 3 (125-cell 3D, FP32 hierarchy, "
                         "rtol 1e-8), 4 (16-cell 2D), 5 (512-cell 256^3, FP32 hierarchy, rtol 1e-8), "
                         "6 (Kir-Na/K 64^3 with a K bolus), 7 (Kir-Na/K 2D), 8 (3D HH, interface-refined grid)")
    ap.add_argument("--nx", type=int, default=None, help="override the mesh resolution of the workload")
    ap.add_argument("--degree", type=int, default=1, choices=[1, 2],
                    help="polynomial degree of the Lagrange elements (2: P2, Section 3.3; with --nx 32 the 3D "
                         "workload has the node lattice of the 64^3 P1 one)")
    ap.add_argument("--adjoint", action="store_true",
                    help="time a checkpointed forward + adjoint run of the 16-cell 2D workload (KNPFunction)")
    args = ap.parse_args()
    if args.config in (3, 5) and "--precision" not in sys.argv:
        args.precision = "fp32"
    if args.config in (3, 5) and "--rtol" not in sys.argv:
        args.rtol = 1e-8
    return args


def workload_name(cfg, n_dof, degree=1):
    membrane = {0: "leak", 1: "HH", 2: "Kir-Na/K"}[cfg.model]
    src = "" if cfg.source_e is None else ", extracellular K bolus / Na removal for x < L/2, 0 < t <= 2 ms"
    el = "" if degree == 1 else ", P2 elements"
    return (f"{cfg.name}: {cfg.dim}D, {cfg.nx}^{cfg.dim} mesh{el}, {len(cfg.cell_lo)} cell(s), {n_dof:,} DOF, "
            f"dt {cfg.dt * 1e3:g} ms, {membrane} membrane{src}")


# --------------------------------------------------------------------------- oracle legs

ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from synth import make_config
from oracle import problem, solve, step, system
cfg = make_config(2).with_nx({nx})
t0 = time.perf_counter()
pb, s = problem.from_config(cfg, degree={degree})
M = solve.lu_P0(system.preconditioner_P0(pb, s))
t_setup = time.perf_counter() - t0
for _ in range({warmup}):
    s, _ = step.step(pb, s, method="gmres", M=M, rtol=1e-13)
times = []
for _ in range({steps}):
    t = time.perf_counter()
    s, _ = step.step(pb, s, method="gmres", M=M, rtol=1e-13)
    times.append(time.perf_counter() - t)
print(json.dumps(dict(n_dof=int(pb.topo.n_dof(3)), setup_s=t_setup, times=times)))
"""


def run_oracle(steps, warmup, nx=SAMPLE_NX, degree=1):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ORACLE_SNIPPET.format(root=ROOT, nx=nx, steps=steps, warmup=warmup, degree=degree)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def oracle_sample_desc(nx, steps, degree=1):
    el = "" if degree == 1 else " with P2 elements"
    return (f"oracle (numpy/scipy FP64, 1 thread) on the same scenario at {nx}^3{el} (same cell, stimulus, dt); "
            f"{steps} steps of assembly + GMRES(30) with LU(P_0) to 1e-13, after 1 untimed step")


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    r = run_oracle(args.steps, args.warmup)
    tot = sum(r["times"])
    value = r["n_dof"] * len(r["times"]) / tot
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * tot / len(r["times"]), higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD + f" (oracle sample at {SAMPLE_NX}^3, {r['n_dof']} DOF)"),
                cpu_baseline=dict(value=value, unit=UNIT, cores=1, kind="oracle",
                                  sample=oracle_sample_desc(SAMPLE_NX, args.steps)),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- our arm

def _source_parts(path, spans):
    src = open(os.path.join(ROOT, "paper_2403_04491_gb300", "csrc", path)).read()
    parts = []
    for start, end in spans:
        a = src.index(start)
        parts.append(src[a:src.index(end, a)])
    return hashlib.sha256("".join(parts).encode()).hexdigest()[:16]


def kernel_source_hash(kind="cheb_fine"):
    """Hash of a reported kernel's source text, so that DRAM counters taken on an older version of
    it are not reported: "cheb_fine" (sell_row, cheb_update, k_cheb_sell) or "spmv" (k_op_apply)."""
    if kind == "spmv":
        return _source_parts("spmv.cu", (("__global__ void __launch_bounds__(128) k_op_apply(",
                                          "// y = rowscale .* (b - A^T x)"),))
    return _source_parts("vcycle.cu", (("// Row product of a sliced-ELL operator", "// Field f of a CSR row product"),
                                       ("// Chebyshev update of one row",
                                        "template <class T, int S>\n__global__ void __launch_bounds__(128) k_cheb_csr")))


def fp64_peak_tflops(torch):
    """Measured FP64 rate of this GPU: best of five 4096^3 DGEMMs (cuBLAS)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None else min(best, t)
    return 2.0 * n ** 3 / best / 1e12


def dominant_kernel_work(prob, precision):
    """Algorithmic bytes and FLOPs of one finest-level Chebyshev step (the V-cycle's largest kernel). Bytes: the operator once
    (column index + four values per stored entry) and six node vectors of four values (x gathered,
    b, D^-1, d read, d written, x written). FLOPs: 4 FMAs per stored entry and 20 per row."""
    info = prob.amg_info()
    n, nnz = info["nodes"][0], info["nnz"][0]
    t = 8 if precision == "fp64" else 4
    return nnz * (4 + 4 * t) + n * 4 * t * 6, 8.0 * nnz + 20.0 * n


def spmv_work(prob):
    """Algorithmic bytes and FLOPs of one operator SpMV y = S^-1 A x (k_op_apply, the Arnoldi
    form without a right-hand side). Bytes: per stored same-region entry a column index and five
    FP64 values (m, a, e^1..e^3), per cross-region entry an index and three values, per node
    the gathered x, the row scale and y (four FP64 each). FLOPs: 9 FMAs per same-region entry,
    3 per cross entry, 20 per row."""
    info = prob.info()
    n, nnz, nx = info["n_nodes"], info["nnz_region"], info["nnz_cross"]
    return nnz * (4 + 40) + nx * (4 + 24) + n * 3 * 32, 18.0 * nnz + 6.0 * nx + 20.0 * n


def measure(prob, torch, steps, rtol, kernel_class=None):
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    from paper_2403_04491_gb300.knp import launch_count
    iters = []
    if kernel_class is not None:
        prob.profile_begin(kernel_class)
    l0 = launch_count()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        iters.append(prob.step(1, rtol=rtol)[0]["iterations"])
    e1.record(stream)
    torch.cuda.synchronize()
    launches = launch_count() - l0
    prof = prob.profile_end() if kernel_class is not None else None
    return e0.elapsed_time(e1), iters, launches, prof


def slowest_rank_ms(ms, world, device):
    """Whole-job time of N replicas: the ranks meet at a barrier and take the largest time."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    dist.barrier()
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def device_memory_gb(torch):
    free, total = torch.cuda.mem_get_info()
    return (total - free) / 1e9


def host_peak_rss_gb():
    """Peak resident host memory of this process so far (mesh generation, topology, setup)."""
    import resource
    return resource.getrusage(resource.RUSAGE_SELF).ru_maxrss * 1024 / 1e9


def job_value(n_dof, steps, world, ms):
    """DOF x steps of all replicas per second of the slowest rank's time."""
    return n_dof * steps * world / (ms / 1e3)


def ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_2403_04491_gb300 import problem_from_config
    from synth import make_config

    cfg = make_config(args.config)
    if args.nx:
        cfg = cfg.with_nx(args.nx)
    prec = 0 if args.precision == "fp64" else 1
    t0 = time.perf_counter()
    mesh, prob = problem_from_config(cfg, degree=args.degree)
    t_create = time.perf_counter() - t0
    t0 = time.perf_counter()
    prob.amg_setup(precision=prec)
    t_amg = time.perf_counter() - t0
    n_dof = prob.n_dof
    free, total = torch.cuda.mem_get_info()
    mem_gb = (total - free) / 1e9
    for _ in range(args.warmup):
        prob.step(1, rtol=args.rtol)
    torch.cuda.synchronize()
    # every measured pass (timed, the two profiled ones, end to end) solves the same steps: the
    # state at the start of the window is restored before each, so iteration counts match
    window = prob.state_get()

    def rewind():
        prob.state_set(window["c_i"], window["phi_i"], window["c_e"], window["phi_e"], window["w"], window["t"])

    if world > 1:
        dist.barrier()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    ms, iters, launches, _ = measure(prob, torch, args.steps, args.rtol)
    clocks = sampler.stop()
    # the reported kernels, timed by per-launch CUDA events on their stream over further passes of
    # the same steps (event pairs go around single launches, so the V-cycle and the Arnoldi steps
    # are not replayed from CUDA graphs in these passes)
    rewind()
    _, _, _, prof = measure(prob, torch, args.steps, args.rtol, kernel_class=1)
    rewind()
    _, _, _, prof_spmv = measure(prob, torch, args.steps, args.rtol, kernel_class=0)
    rewind()
    ms = slowest_rank_ms(ms, world, "cuda")

    # end to end through the public API with host buffers: per step the state goes host->device,
    # one knp_step runs, and the new state comes back device->host (pinned host memory)
    e2e = None if args.no_e2e else e2e_run(prob, torch, args, n_dof, world)
    mixed = None if (args.no_mixed or args.config != 2 or args.degree != 1) else mixed_run(cfg, mesh, torch, args,
                                                                                            n_dof)
    report(args, prob, world, rank, ms, iters, launches, (prof, prof_spmv), clocks, e2e, mixed, n_dof, t_create, t_amg,
           workload_name(cfg, n_dof, args.degree), mem_gb)


def e2e_run(prob, torch, args, n_dof, world):
    import numpy as np
    import torch.distributed as dist
    st = prob.state_get()
    host = {k: torch.from_numpy(np.ascontiguousarray(st[k])).pin_memory() for k in ("c_i", "phi_i", "c_e", "phi_e", "w")}
    dev = {k: torch.empty(v.shape, dtype=torch.float64, device="cuda") for k, v in host.items()}
    h2d = sum(v.numel() * 8 for v in host.values())
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    from paper_2403_04491_gb300 import knp as K
    import ctypes as C
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        for k in host:
            dev[k].copy_(host[k], non_blocking=True)
        ptr = lambda tt: C.cast(C.c_void_p(tt.data_ptr()), K._DP)
        K._check(K._lib.knp_state_set(prob.handle, K.KNP_DEVICE, ptr(dev["c_i"]), ptr(dev["phi_i"]), ptr(dev["c_e"]),
                                      ptr(dev["phi_e"]), ptr(dev["w"]), float(st["t"])))
        prob.step(1, rtol=args.rtol)
        tt = C.c_double()
        K._check(K._lib.knp_state_get(prob.handle, K.KNP_DEVICE, ptr(dev["c_i"]), ptr(dev["phi_i"]), ptr(dev["c_e"]),
                                      ptr(dev["phi_e"]), ptr(dev["w"]), C.byref(tt)))
        st["t"] = tt.value
        for k in host:
            host[k].copy_(dev[k], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_ms = slowest_rank_ms(e2e_ms, world, "cuda")
    e2e_value = job_value(n_dof, args.steps, world, e2e_ms)
    return dict(value=e2e_value, unit=UNIT, h2d_bytes_per_step=h2d, d2h_bytes_per_step=h2d)


def mixed_run(cfg, mesh, torch, args, n_dof):
    """The mixed-precision form (FP32 hierarchy and V-cycle under FP64 FGMRES), same workload."""
    import numpy as np
    from paper_2403_04491_gb300 import problem_from_config
    mixed = None
    if args.precision == "fp64":
        out = {}
        for rt in (1e-10, 1e-8):
            _, pm = problem_from_config(cfg, mesh=mesh)
            pm.amg_setup(precision=1)
            for _ in range(args.warmup):
                pm.step(1, rtol=rt)
            msm, itm, _, _ = measure(pm, torch, args.steps, rt)
            out[f"rtol_{rt:g}"] = dict(value=n_dof * args.steps / (msm / 1e3), iters_per_step=float(np.mean(itm)))
            pm.close()
        _, pf = problem_from_config(cfg, mesh=mesh)
        pf.amg_setup(precision=0)
        for _ in range(args.warmup):
            pf.step(1, rtol=1e-8)
        msf, itf, _, _ = measure(pf, torch, args.steps, 1e-8)
        pf.close()
        out["fp64_rtol_1e-08"] = dict(value=n_dof * args.steps / (msf / 1e3), iters_per_step=float(np.mean(itf)))
        out["speedup_fp32_vs_fp64_at_rtol_1e-08"] = out["rtol_1e-08"]["value"] / out["fp64_rtol_1e-08"]["value"]
        mixed = out
    return mixed


def report(args, prob, world, rank, ms, iters, launches, prof, clocks, e2e, mixed, n_dof, t_create, t_amg,
           workload=WORKLOAD, mem_gb=None):
    import numpy as np
    import torch.distributed as dist
    value = job_value(n_dof, args.steps, world, ms)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    import torch
    p64 = fp64_peak_tflops(torch)
    pf = json.load(open(PROFILE_FILE)) if os.path.exists(PROFILE_FILE) else {}

    def roofline(prof_k, work, key, kind, name, fp64_bound):
        """roofline object of one kernel from its per-launch event timing (n launches, total ms)."""
        n_launch, prof_ms = prof_k
        bytes_per, flops_per = work
        avg_s = prof_ms / n_launch / 1e3 if n_launch else None
        gbs = bytes_per / avg_s / 1e9 if avg_s else None
        ent = pf.get(key)
        # counters hold for the kernel text and the workload they were taken on
        traffic = ent.get("dram_bytes_per_launch") if (ent and ent.get("source_hash") == kernel_source_hash(kind)
                                                       and ent.get("n_dof") == n_dof) else None
        hbm = dict(achieved=gbs, peak=peak, unit="GB/s", frac=(gbs / peak) if gbs else None,
                   peak_source="measured" if "hbm_gbs" in peaks else "fallback")
        common = dict(kernel=name, traffic=traffic, algorithmic_bytes_per_launch=bytes_per,
                      algorithmic_flops_per_launch=flops_per, launches=n_launch,
                      avg_launch_us=1e6 * avg_s if avg_s else None, share_of_step=prof_ms / ms if ms else None)
        if fp64_bound:
            # FP64 arithmetic bounds these kernels on GB300 (FP64 pipe 70-80% busy at about half
            # of HBM, see profiles/): report against the measured FP64 rate, HBM fraction beside it
            tf = flops_per / avg_s / 1e12 if avg_s else None
            return dict(bound="alu", achieved=tf, peak=p64, unit="TFLOP/s", frac=(tf / p64) if tf else None,
                        peak_source="measured FP64 DGEMM 4096^3 in this run", hbm=hbm, **common)
        return dict(bound="hbm", achieved=gbs, peak=peak, unit="GB/s", frac=hbm["frac"],
                    peak_source=hbm["peak_source"], **common)

    # the dominant kernel: the operator SpMV (FP64 in both forms), the largest single kernel of
    # the step (profiles/launches_bench_*); beside it the finest Chebyshev step of the V-cycle
    roof = roofline(prof[1], spmv_work(prob), "spmv_fp64", "spmv",
                    "k_op_apply (operator SpMV S^-1 A x, FP64)", True)
    roof_vc = roofline(prof[0], dominant_kernel_work(prob, args.precision), f"cheb_fine_{args.precision}",
                       "cheb_fine", "k_cheb_sell (finest-level Chebyshev step of the V-cycle)",
                       args.precision == "fp64")
    if mixed and args.precision == "fp64" and args.rtol == 1e-10:
        # the mixed form at its tolerance (1e-8) against the plain FP64 path at its own (1e-10)
        mixed["speedup_fp32_rtol_1e-08_vs_plain_fp64_rtol_1e-10"] = mixed["rtol_1e-08"]["value"] / value
    cpu = None
    if not args.no_baseline and world == 1 and args.config == 2:
        # P2: the sample's mesh is halved, so that its node lattice (and DOF) is the P1 sample's
        snx = SAMPLE_NX if args.degree == 1 else SAMPLE_NX // 2
        r = run_oracle(3, 1, nx=snx, degree=args.degree)
        v = r["n_dof"] * len(r["times"]) / sum(r["times"])
        cpu = dict(value=v, unit=UNIT, cores=1, kind="oracle", sample=oracle_sample_desc(snx, 3, args.degree))
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64" if args.precision == "fp64" else "f64 (FGMRES) / f32 (AMG)", data="synthetic",
                config=dict(workload=workload, n_dof=n_dof, l2="working set per step > L2 (operator, hierarchy and "
                                                               "Krylov basis exceed 129 MB); no flush",
                            precision=args.precision, rtol=args.rtol, restart=30,
                            parallelism=f"replicas x{world}" if world > 1 else "1 GPU"),
                iters_per_step=float(np.mean(iters)), iters=iters, setup_s=dict(create=t_create, amg=t_amg),
                amg=prob.amg_info(), gpu_launches=launches, clocks=clocks, roofline=roof,
                roofline_vcycle=roof_vc,
                device_memory_gb=mem_gb, host_peak_rss_gb=host_peak_rss_gb(),
                e2e=e2e, cpu_baseline=cpu, mixed=mixed)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def adjoint_bench(args):
    """Forward run with checkpoints every 20 steps, then the reverse sweep (recompute + adjoint
    steps), on the differentiation workload; reports both rates and the gradient sizes."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2403_04491_gb300 import KNPFunction, Simulation, problem_from_config, probe_weights
    from synth import make_config
    from synth.configs import probe_points
    # the differentiation workload (4) by default; --config 5 takes the 512-cell 73M-DOF workload
    # (FP32 hierarchy, rtol 1e-8 unless given), whose run asks for one adjoint step (--steps 1)
    cfg = make_config(args.config if "--config" in sys.argv and args.config in (4, 5) else 4)
    if args.nx:
        cfg = cfg.with_nx(args.nx)
    n_steps = args.steps if "--steps" in sys.argv else cfg.n_steps
    rtol = args.rtol if "--rtol" in sys.argv else cfg.rtol
    t0 = time.perf_counter()
    mesh, prob = problem_from_config(cfg)
    prob.amg_setup(precision=1 if cfg.mixed else 0)
    t_setup = time.perf_counter() - t0
    m = cfg.mesh
    ni, ne = mesh.nodes()
    idx, w = probe_weights(m.coords, m.elems, m.elem_tag, ne, prob.N_i, prob.N_e, probe_points(cfg))
    sim = Simulation(prob, idx, w, n_steps, checkpoint_every=20, rtol=rtol, max_it=4000 if cfg.mixed else 1000)
    gK = torch.tensor(prob._facet_gleak[:, 1].copy(), requires_grad=True)
    cK = torch.tensor(sim.s0["c_i"][1].copy(), requires_grad=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    traces = KNPFunction.apply(gK, cK, sim)
    loss = (traces ** 2).sum()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    line = dict(metric="DOF*timesteps/s, forward and checkpointed adjoint", unit="DOF*steps/s", impl="ours",
                config=dict(workload=workload_name(cfg, prob.n_dof) + f", {n_steps} steps, checkpoint every 20, "
                            "loss = sum of phi_e^2 at 64 probes", n_dof=prob.n_dof, rtol=rtol,
                            precision="fp32" if cfg.mixed else "fp64"),
                setup_s=t_setup, device_memory_gb=device_memory_gb(torch), host_peak_rss_gb=host_peak_rss_gb(),
                forward=dict(seconds=t1 - t0, value=prob.n_dof * n_steps / (t1 - t0)),
                adjoint=dict(seconds=t2 - t1, value=prob.n_dof * n_steps / (t2 - t1),
                             note="includes recomputing every segment from its checkpoint"),
                loss=float(loss.detach()), grad_gK_norm=float(gK.grad.norm()), grad_cK_norm=float(cK.grad.norm()),
                iters_forward=sim.its_forward[:5] + (["..."] if len(sim.its_forward) > 5 else []),
                iters_adjoint=sim.its_adjoint[:5] + (["..."] if len(sim.its_adjoint) > 5 else []),
                mean_iters_forward=float(np.mean(sim.its_forward)), mean_iters_adjoint=float(np.mean(sim.its_adjoint)))
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.adjoint:
        adjoint_bench(args)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
