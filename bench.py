#!/usr/bin/env python3
"""Benchmark of the space-time solve on GB300.

One step = one pass of the whole hot path on the 256x256x256 workload (16,974,593
space-time DOFs, extruded Gaussian-random-field design, unit capacity, k ratio 1e-3,
left-edge sink, uniform source): design set-up (Galerkin hierarchy, Jacobi
diagonals, coarsest inverse), forward solve and adjoint solve to a 1e-8 relative
residual with the mixed-precision preconditioner, compliance, and sensitivities.
value = (forward + adjoint DOFs) / step time over all ranks.  Multi-GPU runs are
independent replicas (the solve does not shard across GPUs here).

--impl reference times the FP64 CPU oracle (sparse direct solve) on a bounded
sample of the same workload family on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "space-time DOFs/s to 1e-8 rel. residual, mixed vs FP64; HBM GB/s; p99 latency"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, n in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------- native arm
def run_native(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2508_09589_gb300 import Mesh, lib, options, source
    L = lib()
    w = W.WORKLOADS[args.workload]
    gamma_h = W.make_design(w).reshape(-1)
    layout = "extruded" if w.extruded else "spacetime"
    mesh = Mesh(w.ns, w.nt, material=w.material, bc=w.bc, bc_width=w.bc_width, tau=w.tau, device=local)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    mesh.set_stream(stream.cuda_stream)
    gamma_d = torch.tensor(gamma_h, dtype=torch.float64, device="cuda")
    sens_d = torch.empty_like(gamma_d)
    src = source(w.source, w.source_q0, w.source_a, w.source_b, w.source_f)
    opt = options(rtol=1e-8, precision=args.precision, max_it=400)
    N = mesh.n_nodes

    stats = {}

    def step_device():
        mesh.set_design(gamma_d, layout)
        f = mesh.solve_forward(src, opt)
        phi, a = mesh.solve_adjoint("compliance", opts=opt)
        mesh.sensitivities(sens_d)
        stats.update(fwd=f, adj=a, phi=phi)

    # event timing of the level-0 smoother operator apply inside the solves (event nodes are
    # captured into the V-cycle graphs during warm-up; the totals restart at the timed region)
    mesh.apply_timer(True)
    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()
    barrier(world)
    mesh.apply_timer(True)
    k0 = L.st_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        ev0.record(stream)
        t0 = time.perf_counter()
        its_f, its_a = [], []
        for _ in range(args.steps):
            step_device()
            its_f.append(stats["fwd"]["outer_its"])
            its_a.append(stats["adj"]["outer_its"])
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        torch.cuda.nvtx.range_pop()
    launches = L.st_kernel_launches() - k0
    apply_ms, apply_n = mesh.apply_timer_read()
    mesh.apply_timer(False)
    # the library synchronises its own stream inside each solve, so host wall time brackets
    # all device work of the step; the torch events bracket the same region on the device
    dev_s = max(ev0.elapsed_time(ev1) / 1e3, wall)
    t_step = max_over_ranks(dev_s / args.steps, world)
    barrier(world)
    units = 2.0 * N  # forward + adjoint DOFs per step
    value = units * world / t_step

    # end to end through the C ABI with host buffers (design in, sensitivities out)
    sens_h = np.empty(gamma_h.size)
    e2e_t = []
    for _ in range(max(1, args.steps // 2) if args.e2e else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mesh.set_design(gamma_h, layout)
        mesh.solve_forward(src, opt)
        mesh.solve_adjoint("compliance", opts=opt)
        sens_h = mesh.sensitivities()
        e2e_t.append(time.perf_counter() - t0)
    e2e_step = max_over_ranks(statistics.median(e2e_t), world) if e2e_t else float("nan")

    # all-FP64 comparison arm (one step), mixed vs FP64 at the same 1e-8 outer tolerance
    fp64 = None
    if args.fp64_steps > 0 and args.precision == "mixed":
        opt64 = options(rtol=1e-8, precision="fp64", max_it=400)
        s_mixed = mesh.state("T")
        t64 = []
        for q in range(args.fp64_steps + 1):  # the first step warms the FP64 arm up (graph captures)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mesh.set_design(gamma_d, layout)
            f64 = mesh.solve_forward(src, opt64)
            phi64, a64 = mesh.solve_adjoint("compliance", opts=opt64)
            mesh.sensitivities(sens_d)
            torch.cuda.synchronize()
            if q > 0:
                t64.append(time.perf_counter() - t0)
        s64 = mesh.state("T")
        fp64 = {"value": units / statistics.median(t64), "ms_per_step": 1e3 * statistics.median(t64),
                "steps": len(t64), "warmup": 1, "ms_per_step_samples": [round(1e3 * t, 2) for t in t64],
                "outer_its_fwd": f64["outer_its"], "outer_its_adj": a64["outer_its"],
                "rel_res_fwd": f64["rel_res"], "rel_res_adj": a64["rel_res"],
                "mixed_vs_fp64_rel_T_diff": float(np.abs(s_mixed - s64).max() / np.abs(s64).max())}

    roof = kernel_roofline(N, gamma_h.size if layout == "spacetime" else 0, apply_ms, apply_n, args)
    vc = vcycle_roofline(mesh, args) if (w.extruded and len(w.ns) == 2) else None
    fp64_apply = fp64_apply_roofline(mesh, L, local) if (w.extruded and len(w.ns) == 2) else None

    if rank == 0:
        f, a = stats["fwd"], stats["adj"]
        line = {
            "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "dofs": N, "mesh": list(w.ns) + [w.nt], "precision": args.precision,
                       "rtol": 1e-8, "units": "forward+adjoint DOFs per step",
                       "l2": f"working set {mesh.device_bytes / 1e9:.1f} GB >> 129 MB L2 (no flush needed)",
                       "parallelism": f"replicas x{world}"},
            "forward": {"outer_its": f["outer_its"], "rel_res": f["rel_res"], "seconds": f["seconds"],
                        "ms_per_outer_it": 1e3 * f["seconds"] / max(1, f["outer_its"])},
            "adjoint": {"outer_its": a["outer_its"], "rel_res": a["rel_res"], "seconds": a["seconds"],
                        "ms_per_outer_it": 1e3 * a["seconds"] / max(1, a["outer_its"])},
            "phi": stats["phi"],
            "fp64_arm": fp64,
            "e2e": {"value": units * world / e2e_step, "unit": "DOF/s",
                    "h2d_bytes_per_step": int(gamma_h.nbytes), "d2h_bytes_per_step": int(sens_h.nbytes + 8 * 3)},
            "gpu_launches": int(launches),
            "roofline": roof,
            "vcycle_roofline": vc,
            "fp64_apply_roofline": fp64_apply,
            "clocks": clk.summary(),
        }
    mesh.close()
    if rank == 0:
        # the device-timed line is printed even if one of the auxiliary legs fails
        if args.serve_requests > 0:
            try:
                line["serving"] = serving_bench(args)
            except Exception as e:  # noqa: BLE001
                line["serving"] = {"error": f"{type(e).__name__}: {e}"}
        if args.smoother_variant:
            try:
                line["smoother_variant"] = smoother_variant(args)
            except Exception as e:  # noqa: BLE001
                line["smoother_variant"] = {"error": f"{type(e).__name__}: {e}"}
        if args.example2_iters > 0:
            try:
                line["example2_designs"] = example2_designs(args)
            except Exception as e:  # noqa: BLE001
                line["example2_designs"] = {"error": f"{type(e).__name__}: {e}"}
        if args.design_iters > 0:
            try:
                line["design_loop"] = design_loop(args)
            except Exception as e:  # noqa: BLE001
                line["design_loop"] = {"error": f"{type(e).__name__}: {e}"}
        if args.bdf1:
            try:
                line["bdf1_comparison"] = bdf1_comparison(args)
            except Exception as e:  # noqa: BLE001
                line["bdf1_comparison"] = {"error": f"{type(e).__name__}: {e}"}
        if args.ablation:
            try:
                line["coarsening_ablation"] = coarsening_ablation(args)
            except Exception as e:  # noqa: BLE001
                line["coarsening_ablation"] = {"error": f"{type(e).__name__}: {e}"}
        for name in args.configs:
            try:
                line.setdefault("configs", {})[name] = config_leg(name, args)
            except Exception as e:  # noqa: BLE001
                line.setdefault("configs", {})[name] = {"error": f"{type(e).__name__}: {e}"}
        if args.cpu_baseline:
            try:
                line["cpu_baseline"] = cpu_baseline(args.cpu_sample)
            except Exception as e:  # noqa: BLE001
                line["cpu_baseline"] = {"error": f"{type(e).__name__}: {e}", "kind": "oracle"}
            try:
                line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(args.cpu_sample)
            except Exception as e:  # noqa: BLE001
                line["cpu_baseline_all_cores"] = {"error": f"{type(e).__name__}: {e}", "kind": "oracle"}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def serving_bench(args):
    """Serving stream (the first R requests of the 256-request stream: 2-D + time meshes with
    per-axis element counts log-uniform in 32..512, time 32..256, own seeded designs), each a
    forward + adjoint solve to 1e-8 with sensitivities.  Per precision: a closed-loop run (all
    requests submitted at once) gives the saturation throughput; open-loop runs with Poisson
    arrivals at fractions of that rate give the latency distribution.  The server batches
    queued small requests into shared graph launches (Server max_batch)."""
    import torch
    from paper_2508_09589_gb300 import Server, options, source
    all_reqs = W.serving_requests()
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.85 * free)
    src = source("uniform", 1.0)

    def run(reqs, designs, precision, arrivals, max_batch):
        opt = options(rtol=1e-8, precision=precision, max_it=400)
        srv = Server(budget, max_inflight=args.serve_slots, max_batch=max_batch)
        t0 = time.perf_counter()
        tickets, pending = {}, set()
        k = 0
        res = {}
        while k < len(reqs) or pending:
            now = time.perf_counter() - t0
            while k < len(reqs) and arrivals[k] <= now:
                w = reqs[k]
                tickets[k] = srv.submit(w.ns, w.nt, designs[k], "extruded", src=src, opts=opt,
                                        material=w.material, bc=w.bc, bc_width=w.bc_width)
                pending.add(k)
                k += 1
            for q in list(pending):
                done, r, _ = srv.poll(tickets[q])
                if done:
                    res[q] = r
                    pending.discard(q)
            time.sleep(0.0005)
        span = time.perf_counter() - t0
        srv.close()
        dofs = [(w.ns[0] + 1) * (w.ns[1] + 1) * (w.nt + 1) for w in reqs]
        lat = np.array([res[q]["latency_s"] for q in range(len(reqs))])
        bat = np.array([res[q]["batch"] for q in range(len(reqs))])
        bad = sum(1 for q in range(len(reqs)) if res[q]["status"] != 0)
        return {"requests": len(reqs), "seconds": span, "req_per_s": len(reqs) / span,
                "dof_per_s": 2.0 * sum(dofs) / span,
                "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                "max_ms": 1e3 * float(lat.max()), "failed": bad, "mean_batch": float(bat.mean()),
                "batched_frac": float((bat > 1).mean())}

    out = {"stream": "the 256-request stream (first R requests per precision)", "slots": args.serve_slots,
           "max_batch": args.serve_batch, "hbm_budget_gb": budget / 1e9}
    for precision, nreq, loads in (("mixed", args.serve_requests, args.serve_loads),
                                   ("fp64", args.serve_fp64_requests, args.serve_fp64_loads)):
        if nreq <= 0:
            continue
        reqs = all_reqs[:nreq]
        designs = [W.make_design(w).reshape(-1) for w in reqs]
        leg = {"requests": nreq, "dofs_total": int(sum((w.ns[0] + 1) * (w.ns[1] + 1) * (w.nt + 1) for w in reqs))}
        closed = run(reqs, designs, precision, np.zeros(nreq), args.serve_batch)
        leg["saturation"] = closed
        if args.serve_batch > 1:
            leg["saturation_unbatched"] = run(reqs, designs, precision, np.zeros(nreq), 1)
        for f in loads:
            rate = f * closed["req_per_s"]
            r = run(reqs, designs, precision, W.poisson_arrivals(nreq, rate), args.serve_batch)
            r["offered_req_per_s"] = rate
            leg[f"poisson_{int(round(100 * f))}pct"] = r
        out[precision] = leg
    return out


def step_bytes_per_node(steps: int, tsz: int) -> float:
    """Algorithmic bytes per node of one level-0 Arnoldi-step launch on a stencil level, averaged
    over the steps of a sweep: step 0 reads u_0 and writes w_0; step j >= 1 reads w_{j-1} and
    u_0 .. u_{j-1} and writes u_j and w_j (4 (j + 3) bytes in FP32).  The stencil, with the Jacobi
    scaling folded in, is O(n_x n_y) and stays in L2; the re-reads of u_q for the dot products
    at the node hit L1/L2 (the same block staged them one plane earlier)."""
    per = [2 * tsz] + [tsz * (j + 3) for j in range(1, steps)]
    return float(sum(per)) / steps


def kernel_roofline(N, n_st_elems, apply_ms, apply_n, args, steps=10):
    """Dominant kernel, its launches timed with CUDA events on the mesh stream inside the
    timed steps.  On stencil levels (time-constant 2-D designs) it is the fused Arnoldi step
    km_sm_step (20 launches per V-cycle at level 0, bytes per step_bytes_per_node); on the
    finest level of space-time 2-D designs the marching element apply km_l0st and of extruded
    3-D designs km_l0x3 (w = A D^-1 u: u_j and D^-1 read, w written, 12 B per node in FP32;
    km_l0st also reads the BF16 density, 2 B per space-time element)."""
    peak, kind = _peaks()
    tsz = 4 if args.precision == "mixed" else 8
    if n_st_elems == 0:
        byts = step_bytes_per_node(steps, tsz) * N
    elif n_st_elems < 0:  # extruded 3-D design: the density is O(n_x n_y n_z)
        byts = 3.0 * tsz * N
    else:
        byts = 3.0 * tsz * N + (2.0 * n_st_elems if args.precision == "mixed" else 8.0 * n_st_elems)
    if apply_n <= 0:
        return {"bound": "hbm", "achieved": None, "peak": peak, "unit": "GB/s", "frac": None, "traffic": None}
    t = apply_ms / 1e3 / apply_n
    ach = byts / t / 1e9
    if n_st_elems == 0:
        name, what = "km_sm_step", "fused Arnoldi step: update, stencil apply, dots"
    else:
        name = "km_l0st" if n_st_elems > 0 else "km_l0x3"
        what = "marching smoother operator apply"
    return {"kernel": f"{name} level 0 ({'FP32' if tsz == 4 else 'FP64'} {what})",
            "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": TRAFFIC_PER_LAUNCH.get((name, args.workload, args.precision)),
            "peak_source": kind, "algorithmic_bytes_per_launch": byts, "launch_ms": 1e3 * t,
            "launches_timed": int(apply_n)}


# DRAM read + write bytes of one launch, from an ncu capture of the current kernel version
# (profiles/ names the capture); None when no capture of this version exists.  km_sm_step on
# c1: the mean over the ten level-0 launches j = 0..9 of one sweep (421.1 MB read + 105.4 MB
# written), the same average over j as the achieved bandwidth.
TRAFFIC_PER_LAUNCH = {
    ("km_sm_step", "c1_256x256x256_grf_extruded", "mixed"): 526.5e6,
}


def vcycle_bytes(levels, steps: int, tsz: int) -> float:
    """Algorithmic bytes of one V-cycle on a stencil hierarchy (time-constant 2-D design), each
    vector element read or written once per kernel:
    - pre-smoothing from zero: ||b|| (1 vector), the steps (step_bytes_per_node each), the last
      update (w and the steps basis vectors read, u_steps written), the combination (basis, D^-1
      read, x written);
    - residual (b, x read, r written), restriction (r read, coarse b written), prolongation
      (coarse x read, x read and written);
    - post-smoothing: the start residual (b, x read, u_0 written), the steps, the last update,
      the combination (basis, D^-1, x read, x written);
    - the coarsest level: the dense FP64 inverse (n_c^2 values) and two vectors."""
    per_step = step_bytes_per_node(steps, tsz) * steps
    last_update = tsz * (steps + 2)
    pre = tsz * 1 + per_step + last_update + tsz * (steps + 2)
    post = tsz * 3 + per_step + last_update + tsz * (steps + 3)
    total = 0.0
    for l in range(len(levels) - 1):
        n, nc = levels[l]["n_nodes"], levels[l + 1]["n_nodes"]
        total += (pre + post + 3 * tsz + tsz + 2 * tsz) * n + 2 * tsz * nc
    nc = levels[-1]["n_nodes"]
    total += 8.0 * nc * nc + 2 * tsz * nc
    return total


def vcycle_roofline(mesh, args, cycles: int = 8):
    """One V-cycle of the preconditioner (the operation repeated every outer iteration), timed
    as eager launches through st_vcycle (each call synchronises; the captured graphs of the
    solve run about 1 % faster), against its algorithmic bytes (vcycle_bytes)."""
    import torch
    tsz = 4 if args.precision == "mixed" else 8
    dt = torch.float32 if tsz == 4 else torch.float64
    N = mesh.n_nodes
    g = torch.Generator(device="cuda").manual_seed(7)
    b = torch.randn(N, dtype=dt, device="cuda", generator=g)
    x = torch.empty_like(b)
    mesh.vcycle(b, x, args.precision)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(cycles):
        mesh.vcycle(b, x, args.precision)
    torch.cuda.synchronize()
    t = (time.perf_counter() - t0) / cycles
    byts = vcycle_bytes(mesh.levels(), 10, tsz)
    peak, kind = _peaks()
    return {"ms": 1e3 * t, "algorithmic_bytes": byts, "achieved": byts / t / 1e9, "peak": peak, "unit": "GB/s",
            "frac": byts / t / 1e9 / peak, "peak_source": kind, "cycles": cycles,
            "how": "eager V-cycles through st_vcycle, host-timed with a synchronisation per cycle"}


def fp64_apply_roofline(mesh, L, device: int, reps: int = 10):
    """The FP64 fine operator apply (27-point stencil, 27 FP64 FMAs per node: the outer Krylov
    solver's operator) against the measured FP64 FMA rate of this GPU (st_fp64_fma_rate)."""
    import ctypes as C
    import torch
    N = mesh.n_nodes
    x = torch.randn(N, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    mesh.apply(0, x, y, "fp64")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        mesh.apply(0, x, y, "fp64")
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    peak = C.c_double()
    code = L.st_fp64_fma_rate(device, C.byref(peak))
    tf = 2.0 * 27.0 * N / t / 1e12
    return {"kernel": "km_apply<double> level 0 (FP64 27-point stencil)", "bound": "fp64-alu", "ms": 1e3 * t,
            "achieved": tf, "peak": peak.value if code == 0 else None, "unit": "TFLOP/s",
            "frac": tf / peak.value if code == 0 and peak.value > 0 else None, "flops_per_node": 54,
            "bytes_per_node": 24, "achieved_gbs": 24.0 * N / t / 1e9,
            "peak_source": "measured by st_fp64_fma_rate (independent FMA chains on every SM)"}


def config_leg(name: str, args, steps: int = 1, warmup: int = 1):
    """A further workload timed on its own mesh: set_design, forward and adjoint to 1e-8 and the
    sensitivities, mixed precision (and all-FP64 for one step), with the level-0 smoother
    kernel's CUDA-event roofline."""
    import torch
    from paper_2508_09589_gb300 import Mesh, options, source
    w = W.WORKLOADS[name]
    g = W.make_design(w).reshape(-1)
    layout = "extruded" if w.extruded else "spacetime"
    mesh = Mesh(w.ns, w.nt, material=w.material, bc=w.bc, bc_width=w.bc_width, tau=w.tau)
    src = source(w.source, w.source_q0, w.source_a, w.source_b, w.source_f)
    gd = torch.tensor(g, dtype=torch.float64, device="cuda")
    sens = torch.empty_like(gd)
    N = mesh.n_nodes
    out = {"dofs": N, "mesh": list(w.ns) + [w.nt], "levels": mesh.n_levels}
    for prec, nstep in (("mixed", steps), ("fp64", 1)):
        opt = options(rtol=1e-8, precision=prec, max_it=400)
        if prec == "mixed":
            mesh.apply_timer(True)
        ts = []
        for q in range(warmup + nstep):
            if prec == "mixed" and q == warmup:
                mesh.apply_timer(True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mesh.set_design(gd, layout)
            f = mesh.solve_forward(src, opt)
            phi, a = mesh.solve_adjoint("compliance", opts=opt)
            mesh.sensitivities(sens)
            torch.cuda.synchronize()
            if q >= warmup:
                ts.append(time.perf_counter() - t0)
        t = statistics.median(ts)
        leg = {"value": 2.0 * N / t, "unit": "DOF/s", "ms_per_step": 1e3 * t, "steps": len(ts),
               "forward": {"outer_its": f["outer_its"], "rel_res": f["rel_res"], "seconds": f["seconds"],
                           "dof_per_s": N / f["seconds"]},
               "adjoint": {"outer_its": a["outer_its"], "rel_res": a["rel_res"], "seconds": a["seconds"],
                           "dof_per_s": N / a["seconds"]}}
        if prec == "mixed":
            ms, n = mesh.apply_timer_read()
            mesh.apply_timer(False)
            args_c = argparse.Namespace(precision="mixed", workload=name)
            leg["roofline"] = kernel_roofline(N, g.size if layout == "spacetime" else
                                              (0 if len(w.ns) == 2 else -1), ms, n, args_c)
            s_mixed = mesh.state("T")
        else:
            leg["mixed_vs_fp64_rel_T_diff"] = float(np.abs(s_mixed - mesh.state("T")).max() /
                                                    np.abs(mesh.state("T")).max())
        out[prec] = leg
    out["mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    mesh.close()
    return out


def coarsening_ablation(args):
    """Semi- against full space-time coarsening on the headline workload (the ablation of Sec.
    5.1.2): the same mixed-precision forward + adjoint solve to 1e-8, with every level halving
    space and time together; outer iterations, levels and time of one step after one warm-up."""
    import torch
    from paper_2508_09589_gb300 import Mesh, options, source
    w = W.WORKLOADS[args.workload]
    g = torch.tensor(W.make_design(w).reshape(-1), dtype=torch.float64, device="cuda")
    layout = "extruded" if w.extruded else "spacetime"
    src = source(w.source, w.source_q0, w.source_a, w.source_b, w.source_f)
    opt = options(rtol=1e-8, precision="mixed", max_it=600)
    out = {}
    for mode in ("semi", "full"):
        mesh = Mesh(w.ns, w.nt, material=w.material, bc=w.bc, bc_width=w.bc_width, tau=w.tau, coarsening=mode)
        ts = []
        for q in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mesh.set_design(g, layout)
            f = mesh.solve_forward(src, opt, allow_not_converged=True)
            _, a = mesh.solve_adjoint("compliance", opts=opt, allow_not_converged=True)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        lev = mesh.levels()
        out[mode] = {"levels": len(lev), "coarsest": list(lev[-1]["ns"]) + [lev[-1]["nt"]],
                     "outer_its_fwd": f["outer_its"], "outer_its_adj": a["outer_its"],
                     "converged": bool(f["converged"] and a["converged"]),
                     "ms_per_step": 1e3 * ts[-1], "ms_per_outer_it_fwd": 1e3 * f["seconds"] / max(1, f["outer_its"])}
        mesh.close()
    return out


def smoother_variant(args):
    """The cheaper-smoother variant on the headline workload: the bench's step (set_design,
    forward and adjoint to 1e-8, sensitivities; mixed precision) with damped Jacobi smoothing
    (omega 0.5, nu sweeps) in place of Jacobi-GMRES(10); outer iterations and time of one step
    after one warm-up, for nu = 2 and 4."""
    import torch
    from paper_2508_09589_gb300 import Mesh, options, source
    w = W.WORKLOADS[args.workload]
    g = torch.tensor(W.make_design(w).reshape(-1), dtype=torch.float64, device="cuda")
    layout = "extruded" if w.extruded else "spacetime"
    src = source(w.source, w.source_q0, w.source_a, w.source_b, w.source_f)
    sens = torch.empty_like(g)
    out = {"omega": 0.5}
    mesh = Mesh(w.ns, w.nt, material=w.material, bc=w.bc, bc_width=w.bc_width, tau=w.tau, smoother="jacobi",
                smoother_omega=0.5)
    for nu in (2, 4):
        opt = options(rtol=1e-8, precision="mixed", max_it=600, smooth_steps=nu)
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mesh.set_design(g, layout)
            f = mesh.solve_forward(src, opt, allow_not_converged=True)
            _, a = mesh.solve_adjoint("compliance", opts=opt, allow_not_converged=True)
            mesh.sensitivities(sens)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
        out[f"jacobi_nu{nu}"] = {"ms_per_step": 1e3 * t, "dof_per_s": 2.0 * mesh.n_nodes / t,
                                 "outer_its_fwd": f["outer_its"], "outer_its_adj": a["outer_its"],
                                 "converged": bool(f["converged"] and a["converged"]),
                                 "ms_per_outer_it_fwd": 1e3 * f["seconds"] / max(1, f["outer_its"])}
    mesh.close()
    return out


def example2_designs(args):
    """Example 2 (Sec. 2.3.2) through the optimisation loop: all walls cold, the moving Gaussian
    source (sigma 0.05, radius 0.25, angular frequency pi, tau = 2), v_f = 0.3, an n^2 x n mesh;
    args.example2_iters iterations from gamma = 0.5 at the outer tolerance 1e-5 for an extruded and
    for a space-time design, each final physical design re-evaluated at 1e-8 on a fresh mesh; the
    p-norm temperatures against the homogeneous design of the same volume."""
    from paper_2508_09589_gb300 import Mesh, TopOpt, options, source
    n = args.example2_size
    kw = dict(tau=2.0, material=dict(C_ins=0.5, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3), bc="all_walls",
              bc_width=0.1)
    src = source("gaussian", 1.0, 0.05, 0.25, math.pi)
    tight = options(rtol=1e-8, max_it=300)

    def pnorm_of(design, layout):
        e = Mesh((n, n), n, **kw)
        e.set_design(design, layout)
        e.solve_forward(src, tight)
        phi, _ = e.solve_adjoint("pnorm", P=20, opts=tight)
        e.close()
        return phi
    phi_h = pnorm_of(np.full((n, n), 0.3), "extruded")
    out = {"mesh": [n, n, n], "iterations": args.example2_iters, "phi_homogeneous": phi_h}
    for layout, shape in (("extruded", (n, n)), ("spacetime", (n, n, n))):
        m = Mesh((n, n), n, **kw)
        to = TopOpt(m, np.full(shape, 0.5), layout, vf=0.3)
        t0 = time.perf_counter()
        for _ in range(args.example2_iters):
            to.step(src, options(rtol=1e-5, max_it=200))
        sec = (time.perf_counter() - t0) / max(1, args.example2_iters)
        gb = to.get("gamma_bar")
        to.close()
        m.close()
        phi = pnorm_of(gb, layout)
        out[layout] = {"phi": phi, "ratio_to_homogeneous": phi / phi_h, "chi": float(gb.mean() / 0.3 - 1.0),
                       "s_per_design_iteration": sec}
    return out


def design_loop(args):
    """Design iterations of the optimisation loop (Sec. 3.3) on the headline workload's mesh and
    source: from the homogeneous design gamma = 0.5, v_f = 0.3, the paper's outer tolerance 1e-5
    and warm-started solves; one untimed iteration, then args.design_iters timed ones (wall time
    per iteration, with its forward, adjoint and filter + MMA shares)."""
    from paper_2508_09589_gb300 import Mesh, TopOpt, options, source
    w = W.WORKLOADS[args.design_workload or args.workload]
    mesh = Mesh(w.ns, w.nt, material=w.material, bc=w.bc, bc_width=w.bc_width, tau=w.tau)
    shape = tuple(reversed(w.ns)) if w.extruded else (w.nt,) + tuple(reversed(w.ns))
    to = TopOpt(mesh, np.full(shape, 0.5), "extruded" if w.extruded else "spacetime", vf=0.3)
    src = source(w.source, w.source_q0, w.source_a, w.source_b, w.source_f)
    opt = options(rtol=1e-5, precision="mixed", max_it=200)
    to.step(src, opt)
    its = [to.step(src, opt) for _ in range(args.design_iters)]
    sec = statistics.median(st["seconds"] for st in its)
    fwd = statistics.median(st["forward"]["seconds"] for st in its)
    adj = statistics.median(st["adjoint"]["seconds"] for st in its)
    out = {"workload": w.name, "mesh": list(w.ns) + [w.nt], "design_vars": int(np.prod(shape)),
           "iterations_timed": len(its),
           "ms_per_design_iteration": 1e3 * sec, "forward_ms": 1e3 * fwd, "adjoint_ms": 1e3 * adj,
           "filter_mma_rest_ms": 1e3 * (sec - fwd - adj),
           "filter_ms": 1e3 * statistics.median(st["filter_seconds"] for st in its),
           "projection_set_design_ms": 1e3 * statistics.median(st["design_seconds"] for st in its),
           "mma_ms": 1e3 * statistics.median(st["mma_seconds"] for st in its),
           "outer_its_fwd": [st["forward"]["outer_its"] for st in its],
           "outer_its_adj": [st["adjoint"]["outer_its"] for st in its],
           "filter_cg_its": [st["filter_its"] for st in its],
           "phi": [st["phi"] for st in its], "chi": [st["chi"] for st in its]}
    to.close()
    mesh.close()
    return out


def bdf1_comparison(args):
    """The paper's comparison (Sec. 4) on one GPU: the solves of one design iteration (forward, the
    p-norm adjoint with P = 20, the sensitivities) of the headline workload by the all-at-once
    solver and by the BDF1 time-stepping reference (one FGMRES + spatial multigrid solve per step,
    warm-started from the neighbouring step), both to the paper's outer tolerance 1e-5 in mixed
    precision; one untimed run each, then one timed; the largest difference of the two forward
    trajectories relative to the solution's maximum."""
    import torch
    from paper_2508_09589_gb300 import BDF1, Mesh, options, source
    w = W.WORKLOADS[args.workload]
    g = torch.tensor(W.make_design(w).reshape(-1), dtype=torch.float64, device="cuda")
    layout = "extruded" if w.extruded else "spacetime"
    src = source(w.source, w.source_q0, w.source_a, w.source_b, w.source_f)
    opt = options(rtol=1e-5, precision="mixed", max_it=200)
    kw = dict(material=w.material, bc=w.bc, bc_width=w.bc_width, tau=w.tau)
    sens = torch.empty_like(g)
    mesh = Mesh(w.ns, w.nt, **kw)
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mesh.set_design(g, layout)
        f = mesh.solve_forward(src, opt)
        _, a = mesh.solve_adjoint("pnorm", P=20, opts=opt)
        mesh.sensitivities(sens)
        torch.cuda.synchronize()
        t_st = time.perf_counter() - t0
    Ts = torch.empty(mesh.n_nodes, dtype=torch.float64, device="cuda")
    mesh.state("T", out=Ts)
    out = {"mesh": list(w.ns) + [w.nt], "dofs": mesh.n_nodes,
           "all_at_once": {"ms": 1e3 * t_st, "forward_ms": 1e3 * f["seconds"], "adjoint_ms": 1e3 * a["seconds"],
                           "outer_its_fwd": f["outer_its"], "outer_its_adj": a["outer_its"]}}
    mesh.close()
    b = BDF1(w.ns, w.nt, **kw)
    Tb = torch.empty_like(Ts)
    Lb = torch.empty_like(Ts)
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.set_design(g, layout)
        _, sf = b.forward(src, opt, out=Tb)
        _, _, sa = b.adjoint(20, opt, out=Lb)
        b.sensitivities(sens)
        torch.cuda.synchronize()
        t_b = time.perf_counter() - t0
    b.close()
    out["bdf1"] = {"ms": 1e3 * t_b, "forward_ms": 1e3 * sf["seconds"], "adjoint_ms": 1e3 * sa["seconds"],
                   "steps": sf["steps"], "outer_its_fwd": sf["outer_its"], "outer_its_adj": sa["outer_its"],
                   "max_outer_its_per_step": max(sf["max_outer_its"], sa["max_outer_its"])}
    out["bdf1_over_all_at_once_time"] = t_b / t_st
    out["max_rel_diff_T"] = float((Ts - Tb).abs().max() / Ts.abs().max())
    return out


def run_vcycles(args):
    """Kernel-profiling mode: design set-up and K mixed-precision V-cycles on the workload
    (no Krylov solve, so only the multigrid storage is resident: a few GB at 256^2 x 256)."""
    import torch
    from paper_2508_09589_gb300 import Mesh
    w = W.WORKLOADS[args.workload]
    mesh = Mesh(w.ns, w.nt, material=w.material, bc=w.bc, bc_width=w.bc_width, tau=w.tau)
    mesh.set_design(W.make_design(w).reshape(-1), "extruded" if w.extruded else "spacetime")
    N = mesh.n_nodes
    g = torch.Generator(device="cuda").manual_seed(5)
    b = torch.randn(N, dtype=torch.float32, device="cuda", generator=g)
    x = torch.empty_like(b)
    mesh.vcycle(b, x, "mixed")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.vcycles):
        mesh.vcycle(b, x, "mixed")
    torch.cuda.synchronize()
    t = (time.perf_counter() - t0) / max(1, args.vcycles)
    print(json.dumps({"mode": "vcycles", "workload": w.name, "vcycles": args.vcycles, "ms_per_vcycle": 1e3 * t,
                      "device_gb": mesh.device_bytes / 1e9, "finite": bool(torch.isfinite(x).all())}), flush=True)
    mesh.close()


# ---------------------------------------------------------------------------- oracle (CPU) arm
def cpu_baseline(sample: str):
    """The FP64 oracle as it stands (sparse LU, forward + adjoint) on a bounded sample of
    the workload family, timed on the host cores."""
    from oracle import st_oracle as O
    n = int(sample)
    w = W.scaled(W.C1, (n, n), n)
    om = O.Mesh(w.ns, w.nt, mat=O.Material(**w.material), bc=w.bc, bc_width=w.bc_width)
    g = W.make_design(w)
    t0 = time.perf_counter()
    sol = O.forward(om, g, "uniform", 1.0)
    lam = O.adjoint(sol.A, sol.f, O.dirichlet_mask(om), sol.lu)
    O.sensitivities(om, g, sol.s, lam)
    t = time.perf_counter() - t0
    return {"value": 2.0 * om.n_nodes / t, "unit": "DOF/s", "cores": 1, "kind": "oracle",
            "sample": f"{n}x{n}x{n} mesh of the same family ({om.n_nodes} DOFs), forward+adjoint direct solve "
                      f"(sparse assembly and SuperLU on one core; host has {os.cpu_count()})",
            "seconds": t}


def _oracle_sample(n: int) -> float:
    """Seconds of one oracle sample (used by the all-core baseline's worker processes)."""
    return cpu_baseline(str(n))["seconds"]


def cpu_baseline_all_cores(sample: str):
    """The same oracle sample run as independent problems on every host core at once (one
    process per core, spawned, so no state of the GPU process is inherited): total DOFs
    solved per second of wall time.  SuperLU itself is serial, so this is how the oracle uses
    a many-core host."""
    import multiprocessing as mp
    n = int(sample)
    cores = os.cpu_count() or 1
    w = W.scaled(W.C1, (n, n), n)
    dofs = 2.0 * (n + 1) ** 3
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        secs = pool.map(_oracle_sample, [n] * cores)
    wall = time.perf_counter() - t0
    return {"value": cores * dofs / wall, "unit": "DOF/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} independent {n}x{n}x{n} problems of the same family ({(n + 1) ** 3} DOFs each), "
                      f"forward+adjoint direct solve, one process per core",
            "seconds": wall, "per_problem_seconds_median": statistics.median(secs),
            "workload": w.name}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n = int(args.cpu_sample)
    samples = []
    for q in range(args.warmup + args.steps):
        cb = cpu_baseline(str(n))
        if q >= args.warmup:
            samples.append(cb)
    t = statistics.median(s["seconds"] for s in samples)
    value = statistics.median(s["value"] for s in samples)
    cb = samples[-1]
    line = {"metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": W.C1.name, "sample": cb["sample"]},
            "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=W.C1.name, choices=sorted(W.WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed steps of the all-FP64 arm (after one warm-up)")
    ap.add_argument("--configs", nargs="*", default=["c2_512x512x256_grf_spacetime_sin", "c3_64x64x64x64_grf_extruded_3d"],
                    help="further workloads timed after the headline one (each on its own mesh)")
    ap.add_argument("--cpu-sample", default="34", help="oracle sample n (n^3 mesh, about 10-15 s of CPU work)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-ablation", dest="ablation", action="store_false",
                    help="skip the semi- against full-coarsening comparison")
    ap.add_argument("--serve-requests", type=int, default=96, help="mixed-precision serving requests (0 skips)")
    ap.add_argument("--serve-fp64-requests", type=int, default=48, help="all-FP64 serving requests (0 skips)")
    ap.add_argument("--serve-slots", type=int, default=4, help="server slots (concurrent batches)")
    ap.add_argument("--serve-batch", type=int, default=8, help="requests a slot solves together")
    ap.add_argument("--serve-loads", type=lambda v: [float(x) for x in v.split(",") if x], default=[0.5, 1.0, 1.5],
                    help="Poisson arrival rates as fractions of saturation (mixed precision)")
    ap.add_argument("--serve-fp64-loads", type=lambda v: [float(x) for x in v.split(",") if x], default=[0.7],
                    help="Poisson arrival rates as fractions of saturation (all-FP64)")
    ap.add_argument("--design-workload", default="", choices=[""] + sorted(W.WORKLOADS),
                    help="workload of the design-loop leg (default: --workload)")
    ap.add_argument("--design-iters", type=int, default=3,
                    help="timed design iterations of the optimisation loop after one warm-up (0 skips)")
    ap.add_argument("--example2-iters", type=int, default=0,
                    help="design iterations of the Example 2 leg (extruded against space-time designs; 0 skips)")
    ap.add_argument("--example2-size", type=int, default=128, help="n of the Example 2 leg's n^2 x n mesh")
    ap.add_argument("--smoother-variant", action="store_true",
                    help="also time the damped-Jacobi smoother variant on the headline workload (off by default: "
                         "it does not reach 1e-8 there within 600 outer iterations)")
    ap.add_argument("--no-bdf1", dest="bdf1", action="store_false",
                    help="skip the all-at-once against BDF1 time-stepping comparison")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--vcycles", type=int, default=0,
                    help="profiling mode: only K mixed V-cycles on the workload, no solve")
    args = ap.parse_args()
    if args.vcycles > 0:
        run_vcycles(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
