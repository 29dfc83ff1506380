#!/usr/bin/env python3
"""Benchmark of the KNP-EMI time step (membrane update + assembly + AMG-preconditioned FGMRES).

Default workload: the large mixed-precision scenario, a 256^3 Kuhn mesh of a 100 um cube with an
8 x 8 x 8 array of box cells (side 0.08 L with seeded +-20% jitter, gap 0.03 L), Hodgkin-Huxley
membrane, stimulus 40 S/m^2 on facets with x < 40 um for t < 1 ms, dt = 0.05 ms: 73,078,172
unknowns; AMG hierarchy and V-cycle in FP32 under FP64 FGMRES(30), rtol 1e-8. One "step" is one
IMEX time step; the metric is unknowns x time steps per second. AMG setup (once per run, on P_0)
and topology are excluded, as the paper's "initialization" is; they are reported separately.
Other workloads with --config (2: the 64^3 one-cell FP64 scenario at rtol 1e-10; see --help).

  python bench.py [--gpus N --steps K --warmup W] [--config C] [--impl reference]

Under torchrun (N > 1) every rank runs an independent replica (the path does not shard on
this single-GPU pool); value = unknowns x steps of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import ctypes
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
PROFILE_FILE = os.path.join(ROOT, "profiles", "roofline_counters.json")

# CPU oracle samples per workload: (workload whose scenario the oracle runs, mesh resolution or
# None for the workload's own). The large workloads' cell layouts cannot be coarsened much (their
# cells would touch), so the 512-cell workload takes the 125-cell scenario at 32^3 (192,748
# unknowns), the subset the oracle checks for the mixed-precision workloads.
ORACLE_SAMPLE = {1: (1, None), 2: (2, 24), 3: (3, 32), 4: (4, 64), 5: (3, 32), 6: (6, 24), 7: (7, None),
                 8: (8, 12)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32"],
                    help="hierarchy precision (default: fp32 for the mixed-precision workloads 3 and 5, else fp64)")
    ap.add_argument("--rtol", type=float, default=None, help="FGMRES tolerance (default: the workload's)")
    ap.add_argument("--no-deflate", action="store_true",
                    help="solve without the coarse correction of the potentials' near-null modes")
    ap.add_argument("--no-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--config", type=int, default=5, choices=[1, 2, 3, 4, 5, 6, 7, 8],
                    help="workload: 5 (default: 512-cell 256^3, FP32 hierarchy, rtol 1e-8), 2 (64^3 HH, one "
                         "cell, FP64, rtol 1e-10), 1 (2D leak), 3 (125-cell 128^3, FP32 hierarchy, rtol 1e-8), "
                         "4 (16-cell 2D), 6 (Kir-Na/K 64^3 with a K bolus), 7 (Kir-Na/K 2D), 8 (3D HH, "
                         "interface-refined grid)")
    ap.add_argument("--nx", type=int, default=None, help="override the mesh resolution of the workload")
    ap.add_argument("--degree", type=int, default=1, choices=[1, 2],
                    help="polynomial degree of the Lagrange elements (2: P2, Section 3.3; with --nx 32 the 3D "
                         "workload has the node lattice of the 64^3 P1 one)")
    ap.add_argument("--adjoint", action="store_true",
                    help="time a checkpointed forward + adjoint run of the 16-cell 2D workload (KNPFunction)")
    args = ap.parse_args()
    from synth import make_config
    cfg = make_config(args.config)
    if args.precision is None:
        args.precision = "fp32" if cfg.mixed else "fp64"
    if args.rtol is None:
        args.rtol = cfg.rtol
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
cfg = make_config({cfg_id})
if {nx} is not None:
    cfg = cfg.with_nx({nx})
t0 = time.perf_counter()
pb, s = problem.from_config(cfg, degree={degree})
kw = {{}}
if cfg.dim == 3:
    off_i, off_e, N = system.offsets(pb)
    kw = dict(method="gmres", M=solve.block_lu_P0(system.preconditioner_P0(pb, s), off_i + off_e + [N]), rtol=1e-13)
t_setup = time.perf_counter() - t0
for _ in range({warmup}):
    s, _ = step.step(pb, s, **kw)
times = []
for _ in range({steps}):
    t = time.perf_counter()
    s, _ = step.step(pb, s, **kw)
    times.append(time.perf_counter() - t)
print(json.dumps(dict(n_dof=int(system.offsets(pb)[2]), setup_s=t_setup, times=times)))
"""


def host_cores():
    """Host cores this process may run on (sched_getaffinity), for the CPU oracle replicas."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_replicas(cfg_id, nx, steps, warmup, degree=1, mem_per_replica_gb=6.0):
    """The oracle on every host core at once: one single-threaded process per core, each solving
    the same sample; the rate counts the unknowns x steps of all of them over the slowest one's
    time. Returns (value, cores, n_dof, per-step seconds of the slowest replica)."""
    cores = host_cores()
    try:
        mem_gb = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES") / 1e9
        cores = max(1, min(cores, int(0.7 * mem_gb / mem_per_replica_gb)))
    except (ValueError, OSError, AttributeError):
        pass
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ORACLE_SNIPPET.format(root=ROOT, cfg_id=cfg_id, nx=nx, steps=steps, warmup=warmup, degree=degree)
    procs = [subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for _ in range(cores)]
    outs = []
    for pr in procs:
        o, e = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError(f"oracle replica failed: {e[-2000:]}")
        outs.append(json.loads(o.strip().splitlines()[-1]))
    slowest = max(outs, key=lambda r: sum(r["times"]))
    n_dof = outs[0]["n_dof"]
    value = n_dof * steps * len(outs) / sum(slowest["times"])
    return value, len(outs), n_dof, slowest["times"]


def oracle_sample_desc(cfg_id, nx, steps, warmup, cores, n_dof, degree=1):
    from synth import make_config
    cfg = make_config(cfg_id)
    res = f"{nx}^{cfg.dim}" if nx else f"{cfg.nx}^{cfg.dim}"
    el = "" if degree == 1 else " with P2 elements"
    solver = ("GMRES(30) with the exact LU(P_0) to 1e-13" if cfg.dim == 3 else "sparse LU with refinement")
    return (f"oracle (numpy/scipy FP64) on {cfg.name} at {res}{el} ({n_dof:,} unknowns), {cores} single-threaded "
            f"replicas at once, one per host core; {steps} steps of assembly + {solver} each, after {warmup} "
            f"untimed; rate = all replicas' unknowns x steps / the slowest replica's time")


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg_id, nx = ORACLE_SAMPLE[args.config]
    value, cores, n_dof, times = oracle_replicas(cfg_id, nx, args.steps, args.warmup)
    from synth import make_config
    cfg = make_config(args.config)
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * sum(times) / len(times), higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=f"{cfg.name} (oracle sample: {make_config(cfg_id).name} at "
                                     f"{nx or make_config(cfg_id).nx}, {n_dof:,} DOF)"),
                cpu_baseline=dict(value=value, unit=UNIT, cores=cores, kind="oracle",
                                  sample=oracle_sample_desc(cfg_id, nx, args.steps, args.warmup, cores, n_dof)),
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
        return _source_parts("spmv.cu", (("// w[c] = sum_k z_k tau_r^k x^k[c]",
                                          "// g^k = m + tau_r^k a per stored entry"),))
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
    """Algorithmic bytes and FLOPs of one forward operator product y = S^-1 A x as the library
    times it (the node pass w = sum_k z_k tau^k x^k, then k_op_apply). Bytes: per stored
    same-region entry a column index and seven FP64 values (g^1..g^3 = m + tau^k a, a, e^1..e^3),
    per cross-region entry an index and three values, per node x (4 values) and w read by the
    node pass and w written, then x gathered, w gathered, the row scale and y (FP64). FLOPs: 7 FMAs
    per same-region entry, 3 per cross entry, 3 FMAs per node in the node pass and 20 per row."""
    info = prob.info()
    n, nnz, nx = info["n_nodes"], info["nnz_region"], info["nnz_cross"]
    return nnz * (4 + 56) + nx * (4 + 24) + n * (40 + 104), 14.0 * nnz + 6.0 * nx + 26.0 * n


def measure(prob, torch, steps, rtol, kernel_class=None, deflate=True):
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
        iters.append(prob.step(1, rtol=rtol, deflate=deflate)[0]["iterations"])
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
    defl = not args.no_deflate
    t0 = time.perf_counter()
    mesh, prob = problem_from_config(cfg, degree=args.degree)
    t_create = time.perf_counter() - t0
    t0 = time.perf_counter()
    prob.amg_setup(precision=prec)
    t_amg = time.perf_counter() - t0
    amg_rec = prob.amg_setup_info()
    n_dof = prob.n_dof
    aux = args.steps   # every pass (profiled, end to end, precision comparison) solves the same steps
    for _ in range(args.warmup):
        prob.step(1, rtol=args.rtol, deflate=defl)
    torch.cuda.synchronize()
    # every measured pass (timed, the two profiled ones, end to end) solves steps of the same
    # window: the state at its start is restored before each, so iteration counts match
    window = prob.state_get()

    def rewind(pr):
        pr.state_set(window["c_i"], window["phi_i"], window["c_e"], window["phi_e"], window["w"], window["t"])

    if world > 1:
        dist.barrier()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    ms, iters, launches, _ = measure(prob, torch, args.steps, args.rtol, deflate=defl)
    clocks = sampler.stop()
    mem_gb = device_memory_gb(torch)
    # the reported kernels, timed by per-launch CUDA events on their stream over further passes of
    # the same steps (event pairs go around single launches, so the V-cycle and the Arnoldi steps
    # are not replayed from CUDA graphs in these passes)
    rewind(prob)
    _, _, _, prof = measure(prob, torch, aux, args.rtol, kernel_class=1, deflate=defl)
    rewind(prob)
    _, it_spmv, _, prof_spmv = measure(prob, torch, aux, args.rtol, kernel_class=0, deflate=defl)
    rewind(prob)
    ms = slowest_rank_ms(ms, world, "cuda")
    # end to end through the public API with host buffers: per step the state goes host->device
    # inside knp_state_set(KNP_HOST), one knp_step runs, and knp_state_get(KNP_HOST) brings it back
    e2e = None if args.no_e2e else e2e_run(prob, torch, args, n_dof, world, window, aux, defl)
    rewind(prob)
    work = dict(spmv=spmv_work(prob), cheb=dominant_kernel_work(prob, args.precision), amg=prob.amg_info())
    mixed = None
    if not args.no_mixed and args.degree == 1 and args.config in (2, 3, 5):
        mixed = mixed_run(cfg, mesh, prob, torch, args, n_dof, window, aux, defl)
    prob.close()
    report(args, work, world, rank, ms, iters, launches, (prof, prof_spmv, aux), clocks, e2e, mixed, n_dof,
           t_create, t_amg, amg_rec, workload_name(cfg, n_dof, args.degree), mem_gb, defl)


def e2e_run(prob, torch, args, n_dof, world, window, steps, defl):
    import numpy as np
    from paper_2403_04491_gb300 import knp as K
    host = {k: torch.from_numpy(np.ascontiguousarray(window[k])).pin_memory() for k in ("c_i", "phi_i", "c_e", "phi_e", "w")}
    h2d = sum(v.numel() * 8 for v in host.values())
    ptr = lambda tt: ctypes.cast(ctypes.c_void_p(tt.data_ptr()), K._DP)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t = ctypes.c_double(window["t"])
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        K._check(K._lib.knp_state_set(prob.handle, K.KNP_HOST, ptr(host["c_i"]), ptr(host["phi_i"]),
                                      ptr(host["c_e"]), ptr(host["phi_e"]), ptr(host["w"]), t.value))
        prob.step(1, rtol=args.rtol, deflate=defl)
        K._check(K._lib.knp_state_get(prob.handle, K.KNP_HOST, ptr(host["c_i"]), ptr(host["phi_i"]),
                                      ptr(host["c_e"]), ptr(host["phi_e"]), ptr(host["w"]), ctypes.byref(t)))
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = slowest_rank_ms(e0.elapsed_time(e1), world, "cuda")
    return dict(value=job_value(n_dof, steps, world, e2e_ms), unit=UNIT, h2d_bytes_per_step=h2d,
                d2h_bytes_per_step=h2d, steps=steps,
                path="knp_state_set(KNP_HOST) + knp_step + knp_state_get(KNP_HOST) from pinned host buffers")


def mixed_run(cfg, mesh, prob, torch, args, n_dof, window, steps, defl):
    """The precision comparison on the window's first `steps` steps (setup excluded): the FP32
    hierarchy at rtol 1e-8 (the mixed-precision form), the FP64 hierarchy at 1e-8 (the same
    tolerance), and the plain FP64 path at 1e-10 (the tolerance of the FP64 configs); each
    rate against the others. The timed problem is closed first to free its device memory."""
    import numpy as np
    from paper_2403_04491_gb300 import problem_from_config
    out = {}
    finals = {}
    for key, pr_prec, rt in (("fp32_rtol_1e-08", 1, 1e-8), ("fp64_rtol_1e-08", 0, 1e-8), ("fp64_rtol_1e-10", 0, 1e-10)):
        if pr_prec == (0 if args.precision == "fp64" else 1):
            pm = prob
        else:
            _, pm = problem_from_config(cfg, mesh=mesh)
            pm.amg_setup(precision=pr_prec)
        pm.state_set(window["c_i"], window["phi_i"], window["c_e"], window["phi_e"], window["w"], window["t"])
        msm, itm, _, _ = measure(pm, torch, steps, rt, deflate=defl)
        out[key] = dict(value=n_dof * steps / (msm / 1e3), iters_per_step=float(np.mean(itm)), iters=itm)
        st = pm.state_get()
        finals[key] = (np.concatenate([st["c_i"].ravel(), st["c_e"].ravel()]), np.concatenate([st["phi_i"], st["phi_e"]]))
        if pm is not prob:
            pm.close()
    out["steps"] = steps

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    # the mixed form's states after the window's steps against the FP64 GPU path's (at 1e-8 and
    # at 1e-10), relative l2 over the concentrations and over the potentials
    for ref_key in ("fp64_rtol_1e-08", "fp64_rtol_1e-10"):
        out[f"fp32_rtol_1e-08_vs_{ref_key}"] = dict(
            rel_diff_c=rel(finals["fp32_rtol_1e-08"][0], finals[ref_key][0]),
            rel_diff_phi=rel(finals["fp32_rtol_1e-08"][1], finals[ref_key][1]))
    out["speedup_fp32_vs_fp64_at_rtol_1e-08"] = out["fp32_rtol_1e-08"]["value"] / out["fp64_rtol_1e-08"]["value"]
    out["speedup_fp32_rtol_1e-08_vs_plain_fp64_rtol_1e-10"] = (out["fp32_rtol_1e-08"]["value"]
                                                               / out["fp64_rtol_1e-10"]["value"])
    return out


def report(args, work, world, rank, ms, iters, launches, prof, clocks, e2e, mixed, n_dof, t_create, t_amg, amg_rec,
           workload, mem_gb, defl):
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
    aux = prof[2]
    ms_aux = ms * aux / args.steps   # the profiled passes cover the window's first `aux` steps

    def roofline(prof_k, work_k, key, kind, name, fp64_bound):
        """roofline object of one kernel from its per-launch event timing (n launches, total ms)."""
        n_launch, prof_ms = prof_k
        bytes_per, flops_per = work_k
        avg_s = prof_ms / n_launch / 1e3 if n_launch else None
        gbs = bytes_per / avg_s / 1e9 if avg_s else None
        ent = pf.get(key)
        # counters hold for the kernel text they were taken on: as captured on the same workload,
        # else scaled by the algorithmic bytes (the capture's traffic / algorithmic ratio)
        traffic, traffic_src = None, None
        if ent and ent.get("source_hash") == kernel_source_hash(kind):
            if ent.get("n_dof") == n_dof:
                traffic, traffic_src = ent.get("dram_bytes_per_launch"), "ncu capture of this workload"
            elif ent.get("algorithmic_bytes_per_launch"):
                traffic = ent["dram_bytes_per_launch"] / ent["algorithmic_bytes_per_launch"] * bytes_per
                traffic_src = (f"scaled by algorithmic bytes from the ncu capture at {ent['n_dof']:,} DOF "
                               f"(traffic / algorithmic = {ent['dram_bytes_per_launch'] / ent['algorithmic_bytes_per_launch']:.3f})")
        hbm = dict(achieved=gbs, peak=peak, unit="GB/s", frac=(gbs / peak) if gbs else None,
                   peak_source="measured" if "hbm_gbs" in peaks else "fallback")
        common = dict(kernel=name, traffic=traffic, traffic_source=traffic_src, algorithmic_bytes_per_launch=bytes_per,
                      algorithmic_flops_per_launch=flops_per, launches=n_launch,
                      avg_launch_us=1e6 * avg_s if avg_s else None,
                      share_of_step=prof_ms / ms_aux if ms_aux else None)
        if fp64_bound:
            # FP64 arithmetic bounds these kernels on GB300 (its FP64 pipe is 1/64 of FP32): report
            # against the measured FP64 rate, the HBM fraction beside it
            tf = flops_per / avg_s / 1e12 if avg_s else None
            return dict(bound="alu", achieved=tf, peak=p64, unit="TFLOP/s", frac=(tf / p64) if tf else None,
                        peak_source="measured FP64 DGEMM 4096^3 in this run", hbm=hbm, **common)
        return dict(bound="hbm", achieved=gbs, peak=peak, unit="GB/s", frac=hbm["frac"],
                    peak_source=hbm["peak_source"], **common)

    # the dominant kernel: the operator SpMV (FP64 in both forms); beside it the finest Chebyshev
    # step of the V-cycle
    roof = roofline(prof[1], work["spmv"], "spmv_fp64", "spmv", "k_op_apply (operator SpMV S^-1 A x, FP64)", True)
    roof_vc = roofline(prof[0], work["cheb"], f"cheb_fine_{args.precision}", "cheb_fine",
                       "k_cheb_sell (finest-level Chebyshev step of the V-cycle)", args.precision == "fp64")
    cpu = None
    if not args.no_baseline and world == 1:
        cfg_id, nx = ORACLE_SAMPLE[args.config]
        if args.degree == 2 and nx:
            nx //= 2   # P2: the sample's mesh is halved, so that its node lattice is the P1 sample's
        v, cores, sdof, _ = oracle_replicas(cfg_id, nx, 3, 1, degree=args.degree)
        cpu = dict(value=v, unit=UNIT, cores=cores, kind="oracle",
                   sample=oracle_sample_desc(cfg_id, nx, 3, 1, cores, sdof, args.degree))
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64" if args.precision == "fp64" else "f64 (FGMRES) / f32 (AMG)", data="synthetic",
                config=dict(workload=workload, n_dof=n_dof, l2="working set per step > L2 (operator, hierarchy and "
                                                               "Krylov basis exceed 129 MB); no flush",
                            precision=args.precision, rtol=args.rtol, restart=30, deflate=defl,
                            parallelism=f"replicas x{world}" if world > 1 else "1 GPU"),
                iters_per_step=float(np.mean(iters)), iters=iters, setup_s=dict(create=t_create, amg=t_amg),
                amg=work["amg"], amg_setup=amg_rec, gpu_launches=launches, clocks=clocks, roofline=roof,
                roofline_vcycle=roof_vc, profiled_steps=aux,
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
    max_it = 4000 if cfg.mixed else 1000
    sim = Simulation(prob, idx, w, n_steps, checkpoint_every=20, rtol=rtol, max_it=max_it)
    # warm-up: a short forward and reverse sweep from the same initial state, so that the timed run
    # does not pay the first use of each kernel, graph and work array (the first forward of a
    # fresh process took 3.8 s more than the same forward repeated, on the 200-step 2D workload)
    warm = Simulation(prob, idx, w, max(1, args.warmup), checkpoint_every=20, rtol=rtol, max_it=max_it)
    gKw = torch.tensor(prob._facet_gleak[:, 1].copy(), requires_grad=True)
    cKw = torch.tensor(warm.s0["c_i"][1].copy(), requires_grad=True)
    (KNPFunction.apply(gKw, cKw, warm) ** 2).sum().backward()
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
                setup_s=t_setup, warmup_steps=max(1, args.warmup), device_memory_gb=device_memory_gb(torch),
                host_peak_rss_gb=host_peak_rss_gb(),
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
