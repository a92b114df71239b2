#!/usr/bin/env python3
"""Benchmark: semi-implicit BDF2 VMS-LES Navier-Stokes steps per second on a ~1M-tetrahedron
cylinder (Poiseuille set-up: R = 1 cm, L = 10 cm, blood rho = 1.06, mu = 0.035, parabolic inlet
ramped to a 20 cm/s peak, zero-traction outlet, dt = 1e-3 s), synthetic seeded mesh.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle on a bounded sample
of the same workload instead.  With --gpus N > 1 (torchrun), every rank runs its own
independent simulation (replicas; the method does not exchange data between them).
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

R_CM, L_CM, U_PEAK, RHO, MU, DT = 1.0, 10.0, 20.0, 1.06, 0.035, 1e-3
RAMP = 0.05                      # s, sinusoidal ramp of the inflow (Section 2.2.1)
L2_BYTES = 129 * 2 ** 20
FP64_PEAK_TFLOPS = 1.20            # measured FP64 FMA-throughput probe on a GB300 (nvcc-built, run once)
FP32_ISSUE_PEAK_T = 35.96          # measured FP32 FMA-issue probe on a GB300, T thread-instructions/s
# FP64-class operations of the method per tetrahedron (DFMA x 2 + DADD + DMUL executed by the FP64
# assembly kernel, counted with ncu): the algorithmic work of one element's assembly
ASM_FP64_FLOPS_PER_ELEMENT = 2948
# thread instructions per tetrahedron of the double-float assembly kernel (ncu) and its DRAM
# bytes per tetrahedron (ncu, one colour launch of 29,184 elements; profiles/)
ASM_DD_INST_PER_ELEMENT = 28477
ASM_DD_DRAM_BYTES_PER_ELEMENT = 4331
# DRAM bytes per block of the FP32 Krylov SpMV (ncu read + write, 2,089,595-block launch)
SPMV32_DRAM_BYTES_PER_BLOCK = 71.6


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    def __init__(self):
        self.samples, self.proc = [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        dev = os.environ.get("LOCAL_RANK", "0")
        rows = [s for s in self.samples if s and s[0] == dev] or self.samples
        sm = [float(s[1]) for s in rows if len(s) > 8 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in rows if len(s) > 8 and s[2].replace(".", "").isdigit()]
        reasons = set()
        for s in rows:
            if len(s) > 8:
                for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                                   s[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def make_case(n_tets, seed=2):
    from synthetic import cylinder

    t0 = time.time()
    m = cylinder(R_CM, L_CM, n_tets=n_tets, seed=seed)
    return m, time.time() - t0


def gpu_problem(L, m, precision):
    Q = U_PEAK * math.pi * R_CM ** 2 / 2.0
    bcs = [L.BC(tag=0, kind="noslip"),
           L.BC(tag=1, kind="dirichlet", profile="parabolic", time="ramp", p=(0.0, Q, 0.0, RAMP), radius=R_CM),
           L.BC(tag=2, kind="neumann", time="constant", p=(0.0,))]
    extra = dict(smoother_bf16=1) if precision == "mixed" else {}
    opts = L.default_options(precision=precision, gmres_rtol=1e-8, **extra)
    mesh = L.Mesh.from_synthetic(m)
    prob = L.Problem(mesh, RHO, MU, DT, 2, bcs, [], opts)
    return mesh, prob


def replica_throughput(ms_local, steps, dist=None, device=None):
    """Whole-job throughput of independent replicas (one simulation per rank, no data exchange):
    the slowest rank's time bounds the job, every rank contributes `steps` steps."""
    import torch

    world = dist.get_world_size() if dist is not None else 1
    ms = ms_local
    if dist is not None:
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * steps / (ms * 1e-3), ms


def timed_steps(L, st, steps, warmup, stream):
    import torch

    for _ in range(warmup):
        st.step(allow_not_converged=True)
    torch.cuda.synchronize()
    n0 = L.library().lfx_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = [st.step(allow_not_converged=True) for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), stats, L.library().lfx_launch_count() - n0


def run_gpu(args):
    import torch

    from paper_2304_12032_gb300 import build as B

    B.build()
    from paper_2304_12032_gb300 import lfx as L

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    m, tgen = make_case(args.tets, seed=2 + rank)
    V = m.n_nodes
    stream = torch.cuda.current_stream()
    # common starting state: the FP64 path run through the warm-up steps from rest
    mesh64, prob64 = gpu_problem(L, m, "fp64")
    st64 = L.State(prob64, np.zeros((2, V, 3)), np.zeros((2, V)), 0.0, stream=stream)
    for _ in range(args.warmup):
        st64.step(allow_not_converged=True)
    u1, p1 = st64.get()
    # history level 1 from a second FP64 step snapshot is not kept by the API: restart BDF2 from
    # two copies of the warm state
    hist_u, hist_p, t_start = np.stack([u1, u1]), np.stack([p1, p1]), args.warmup * DT
    results = {}
    for prec in (["mixed", "fp64"] if args.precision == "both" else [args.precision]):
        mesh, prob = (mesh64, prob64) if prec == "fp64" else gpu_problem(L, m, prec)
        st = L.State(prob, hist_u, hist_p, t_start, stream=stream)
        if dist:
            dist.barrier()
        clocks = Clocks()
        clocks.start()
        ms, stats, launches = timed_steps(L, st, args.steps, 1, stream)
        clk = clocks.stop()
        _, ms = replica_throughput(ms, args.steps, dist, "cuda")
        u, p = st.get()
        results[prec] = dict(ms=ms, stats=stats, launches=launches, clocks=clk, u=u, p=p, st=st, mesh=mesh)
    prim = results["mixed"] if "mixed" in results else results[args.precision]
    prim_prec = "mixed" if "mixed" in results else args.precision
    info = prim["mesh"].info()
    st = prim["st"]
    # ---- end to end through the public API: host history in, solution out, every step
    # (inputs and results in page-locked host buffers, which the copies read and write by DMA)
    sigma = 2

    def pinned(*shape):
        return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()

    hu, hp = pinned(sigma, V, 3), pinned(sigma, V)
    hu[:] = prim["u"]
    hp[:] = prim["p"]
    u_host, p_host = pinned(V, 3), pinned(V)
    t_now = prim["stats"][-1]["t"]
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for k in range(args.steps):
        st.set(hu, hp, t_now)
        st.step(allow_not_converged=True)
        st.get(u_host, p_host)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - w0) * 1e3 / args.steps
    h2d, d2h = 2 * V * 4 * 8, V * 4 * 8
    # ---- rooflines from CUDA events recorded inside the timed steps (on the state's stream)
    stats = prim["stats"]
    T, nnzb = info["n_tets"], info["nnz_blocks"]
    peaks, src = _peaks()
    spmv_ms = sum(s["ms_spmv"] for s in stats) / max(1, sum(s["n_spmv"] for s in stats))
    sv = 4 if prim_prec == "mixed" else 8            # inner Krylov matrix / vector precision
    spmv_bytes = nnzb * (16 * sv + 4) + 4 * (V + 1) + 2 * 4 * V * sv
    spmv_bw = spmv_bytes / (spmv_ms * 1e-3) / 1e9
    roof = {"kernel": f"spmv_kernel ({'FP32' if sv == 4 else 'FP64'} 4x4 block CSR, Arnoldi products)",
            "bound": "hbm", "achieved": round(spmv_bw, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(spmv_bw / peaks["hbm_gbs"], 4),
            "traffic": int(SPMV32_DRAM_BYTES_PER_BLOCK * nnzb) if sv == 4 else None, "peak_source": src + " (burst copy)",
            "ms_per_launch": round(spmv_ms, 4), "launches_timed": int(sum(s["n_spmv"] for s in stats)),
            "algorithmic_bytes_per_launch": int(spmv_bytes)}
    asm_ms = sum(s["ms_assembly_kernels"] for s in stats) / len(stats)
    n_asm = stats[0]["n_assembly_launches"]
    asm_bytes = 16 * T + V * (3 * 8 + 8 * 8) + nnzb * 16 * 8 + 4 * V * 8
    asm_flops = ASM_FP64_FLOPS_PER_ELEMENT * T
    if prim_prec == "mixed":
        # double-float assembly: bounded by FP32 instruction issue (FMA pipe), not by HBM
        inst_rate = ASM_DD_INST_PER_ELEMENT * T / (asm_ms * 1e-3) / 1e12
        roof_asm = {"kernel": "assemble_color_kernel<dd> (double-float arithmetic on the FP32 pipes; all colours of one step)",
                    "bound": "alu", "achieved": round(inst_rate, 3), "peak": FP32_ISSUE_PEAK_T,
                    "unit": "T thread-inst/s", "frac": round(inst_rate / FP32_ISSUE_PEAK_T, 4),
                    "traffic": int(ASM_DD_DRAM_BYTES_PER_ELEMENT * T / n_asm),
                    "peak_source": "measured FP32 FMA-issue probe (nvcc-built, run once on a GB300)",
                    "inst_per_element": ASM_DD_INST_PER_ELEMENT,
                    "fp64_class_tflops": round(asm_flops / (asm_ms * 1e-3) / 1e12, 4),
                    "fp64_class_flops_per_element": ASM_FP64_FLOPS_PER_ELEMENT,
                    "hbm_view": {"achieved_gbs": round(asm_bytes / (asm_ms * 1e-3) / 1e9, 1),
                                 "algorithmic_bytes": int(asm_bytes)},
                    "ms_per_step": round(asm_ms, 4), "ms_per_launch": round(asm_ms / n_asm, 4),
                    "launches_per_step": n_asm}
    else:
        roof_asm = {"kernel": "assemble_color_kernel<double> (all colours of one step)", "bound": "alu",
                    "achieved": round(asm_flops / (asm_ms * 1e-3) / 1e12, 4), "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": round(asm_flops / (asm_ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, 4),
                    "traffic": None, "peak_source": "measured FP64 FMA probe (nvcc-built, run once on a GB300)",
                    "hbm_view": {"achieved_gbs": round(asm_bytes / (asm_ms * 1e-3) / 1e9, 1),
                                 "algorithmic_bytes": int(asm_bytes)},
                    "ms_per_step": round(asm_ms, 4), "ms_per_launch": round(asm_ms / n_asm, 4),
                    "launches_per_step": n_asm, "fp64_flops_per_element": ASM_FP64_FLOPS_PER_ELEMENT}
    its = [s["iterations"] for s in stats]
    ms = prim["ms"]
    value = world * args.steps / (ms * 1e-3)
    line = {
        "metric": "time steps/s at 1M P1 tets (BDF2 VMS-LES step: assembly + aSIMPLE-GMRES)",
        "value": round(value, 3), "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prim_prec == "fp64" else "f32+f64",
        "data": "synthetic (seeded jittered-BCC Delaunay cylinder; no paper meshes available)",
        "config": {"workload": f"poiseuille_cylinder_{T}_tets", "n_tets": T, "n_nodes": V, "nnz_blocks": nnzb,
                   "n_colors": info["n_colors"], "precision": prim_prec, "bdf_order": 2, "dt": DT,
                   "gmres_rtol": 1e-8, "krylov_iterations_mean": statistics.mean(its),
                   "outer_iterations_mean": statistics.mean(s["outer_iterations"] for s in stats),
                   "l2": "inputs larger than L2 (FP64 matrix %.0f MB > 129 MB)" % (nnzb * 16 * 8 / 1e6),
                   "mesh_gen_s": round(tgen, 1), "start": f"from rest, {args.warmup} FP64 warm-up steps"},
        "elements_per_s_assembly": round(T / (asm_ms * 1e-3), 1),
        "phase_ms": {"assembly": round(statistics.mean(s["ms_assembly"] for s in stats), 3),
                     "solve": round(statistics.mean(s["ms_solve"] for s in stats), 3)},
        # the dominant kernel of the step is the assembly (one launch per colour); the Krylov SpMV
        # is the dominant HBM-bound kernel
        "roofline": roof_asm,
        "roofline_spmv": roof,
        "e2e": {"value": round(1e3 / e2e_ms * world, 3), "unit": "steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(prim["launches"]),
        "clocks": prim["clocks"],
    }
    if "fp64" in results and prim_prec != "fp64":
        r64 = results["fp64"]
        v64 = world * args.steps / (r64["ms"] * 1e-3)
        du = np.linalg.norm(prim["u"] - r64["u"]) / np.linalg.norm(r64["u"])
        dp = np.linalg.norm(prim["p"] - r64["p"]) / np.linalg.norm(r64["p"])
        line["fp64_gpu"] = {"value": round(v64, 3), "unit": "steps/s", "ms_per_step": round(r64["ms"] / args.steps, 3),
                            "krylov_iterations_mean": statistics.mean(s["iterations"] for s in r64["stats"]),
                            "gpu_launches": int(r64["launches"])}
        line["speedup_mixed_vs_fp64"] = round(value / v64, 3)
        line["mixed_vs_fp64_rel_l2_after_steps"] = {"u": float(du), "p": float(dp)}
    if rank == 0 and args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_sample_tets)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_serving(args):
    """Serving workload (continuous batching): Poisson arrivals (mean args.rate req/s) of
    simulations on cylinder / stenosis geometries drawn from a pre-generated pool (sizes
    log-uniform in [args.serve_min, args.serve_max] tets), each asking for args.req_steps BDF2
    steps, admitted by a device-memory budget into the native request loop.  Reports p50/p99
    per-step latency and aggregate steps/s, beside the same requests run back to back on one
    stream (sequential FP64 GPU)."""
    import torch

    from paper_2304_12032_gb300 import build as B

    B.build()
    from paper_2304_12032_gb300 import lfx as L
    from synthetic import stenosis

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rng = np.random.default_rng(5)
    sizes = np.exp(np.linspace(math.log(args.serve_min), math.log(args.serve_max), args.pool))
    pool = []
    Q = U_PEAK * math.pi * R_CM ** 2 / 2.0
    for i, nt in enumerate(sizes):
        m = make_case(int(nt), seed=50 + i)[0] if i % 2 == 0 else stenosis(R_CM, L_CM, n_tets=int(nt), seed=50 + i)
        bcs = [L.BC(tag=0, kind="noslip"),
               L.BC(tag=1, kind="dirichlet", profile="parabolic", time="ramp", p=(0.0, Q, 0.0, RAMP), radius=R_CM),
               L.BC(tag=2, kind="neumann", time="constant", p=(0.0,))]
        mesh = L.Mesh.from_synthetic(m)
        prob = L.Problem(mesh, RHO, MU, DT, 2, bcs, [], L.default_options(
            gmres_rtol=1e-8, precision=args.serve_precision, **({"smoother_bf16": 1} if args.serve_precision == "mixed" else {})))
        prob64 = prob if args.serve_precision == "fp64" else L.Problem(mesh, RHO, MU, DT, 2, bcs, [], L.default_options(gmres_rtol=1e-8))
        pool.append((m, mesh, prob, prob64))
    free = torch.cuda.mem_get_info()[0]
    budget = int(args.serve_budget_frac * free)
    n_req = max(1, int(round(args.rate * args.serve_seconds)))
    gaps = rng.exponential(1.0 / args.rate, n_req)
    picks = rng.integers(0, len(pool), n_req)
    srv = L.Server(budget, n_workers=args.workers)
    t0 = time.perf_counter()
    tickets, submit_t = [], []
    arrival = 0.0
    for k in range(n_req):
        arrival += gaps[k]
        while time.perf_counter() - t0 < arrival:
            time.sleep(0.001)
        m, mesh, prob, _ = pool[picks[k]]
        V = m.n_nodes
        tickets.append(srv.submit(prob, np.zeros((2, V, 3)), np.zeros((2, V)), 0.0, args.req_steps))
        submit_t.append(time.perf_counter() - t0)
    while not all(srv.poll(t)[0] for t in tickets):
        time.sleep(0.01)
    wall = time.perf_counter() - t0
    st = srv.stats()
    for t in tickets:
        srv.result(t)
    srv.close()
    lat = st["latency_ms"]
    total_steps = n_req * args.req_steps
    # sequential FP64 GPU: every distinct pool entry stepped alone, scaled by how often it was picked
    seq_ms = 0.0
    for j, (m, mesh, _, prob64) in enumerate(pool):
        cnt = int(np.sum(picks == j))
        if cnt == 0:
            continue
        s1 = L.State(prob64, np.zeros((2, m.n_nodes, 3)), np.zeros((2, m.n_nodes)), 0.0)
        s1.step(allow_not_converged=True)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for _ in range(min(args.req_steps, 10)):
            s1.step(allow_not_converged=True)
        torch.cuda.synchronize()
        seq_ms += (time.perf_counter() - w0) * 1e3 / min(args.req_steps, 10) * args.req_steps * cnt
    line = {"metric": "serving: per-step latency p50/p99 and aggregate steps/s (continuous batching)",
            "value": round(total_steps / wall, 2), "unit": "steps/s", "n_gpus": 1,
            "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "requests": n_req, "steps_per_request": args.req_steps, "wall_s": round(wall, 2),
            "sequential_fp64_steps_per_s": round(total_steps / (seq_ms * 1e-3), 2),
            "speedup_vs_sequential": round((total_steps / wall) / (total_steps / (seq_ms * 1e-3)), 3),
            "max_resident": st["max_active"], "budget_bytes": budget, "workers": args.workers,
            "pool_tets": [int(p[0].n_tets) for p in pool], "arrival_rate_req_s": args.rate,
            "higher_is_better": True, "dtype": "f32+f64" if args.serve_precision == "mixed" else "f64",
            "precision": args.serve_precision, "data": "synthetic"}
    print(json.dumps(line), flush=True)


def run_batched(args):
    """Batched workload: args.batch independent pipe and Y-bifurcation meshes of seeded
    sizes uniform in [args.batch_min, args.batch_max] tets, stepped as ONE system (one coloured
    assembly launch per colour; one Krylov solve for all of them with one Arnoldi process per
    mesh, sharing every launch; per-mesh row normalisation), against the same meshes stepped one
    after another (FP64 GPU and mixed), and against the union solved as a single Krylov system."""
    import torch

    from paper_2304_12032_gb300 import build as B

    B.build()
    from paper_2304_12032_gb300 import lfx as L
    from synthetic import batch, bifurcation, cylinder

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rng = np.random.default_rng(4)
    t0 = time.time()
    ms = []
    for i in range(args.batch):
        nt = int(rng.uniform(args.batch_min, args.batch_max))
        if i % 2 == 0:
            r = float(rng.uniform(0.3, 1.2))
            ms.append(cylinder(r, 8.0 * r, n_tets=nt, seed=1000 + i))
        else:
            s_ = float(rng.uniform(0.3, 1.2)) / 0.6
            ms.append(bifurcation(n_tets=nt, seed=1000 + i, angle_deg=float(rng.uniform(30, 70)),
                                  r0=0.6 * s_, r1=0.45 * s_, r2=0.4 * s_))
    tgen = time.time() - t0

    def member_bcs(i, m, stride):
        out = [L.BC(tag=0 + stride * i, kind="noslip")]
        if "radius" in m.meta:
            R = m.meta["radius"]
            Q = U_PEAK * math.pi * R * R / 2.0
            out.append(L.BC(tag=1 + stride * i, kind="dirichlet", profile="parabolic", time="ramp",
                            p=(0.0, Q, 0.0, RAMP), radius=R))
        else:
            out.append(L.BC(tag=1 + stride * i, kind="dirichlet", profile="uniform", time="ramp",
                            p=(0.0, U_PEAK / 2.0, 0.0, RAMP)))
        for t in sorted(set(np.unique(m.btags).tolist()) - {0, 1}):
            out.append(L.BC(tag=int(t) + stride * i, kind="neumann", time="constant", p=(0.0,)))
        return out

    def steps_time(mesh_syn, bcs, precision, n, segmented=1):
        opts = L.default_options(precision=precision, gmres_rtol=1e-8, batch_segmented=segmented,
                                 **({"smoother_bf16": 1} if precision == "mixed" else {}))
        prob = L.Problem(L.Mesh.from_synthetic(mesh_syn), RHO, MU, DT, 2, bcs, [], opts)
        V = mesh_syn.n_nodes
        st = L.State(prob, np.zeros((2, V, 3)), np.zeros((2, V)), 0.0)
        for _ in range(args.warmup):
            st.step(allow_not_converged=True)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        its = [st.step(allow_not_converged=True)["iterations"] for _ in range(n)]
        torch.cuda.synchronize()
        return (time.perf_counter() - w0) / n, its

    u = batch(ms)
    bcs = sum((member_bcs(i, m, 10) for i, m in enumerate(ms)), [])
    t_batch, its_b = steps_time(u, bcs, "mixed", args.steps)
    t_union, its_u = steps_time(u, bcs, "mixed", max(2, args.steps // 2), segmented=0)
    seq = {"fp64": 0.0, "mixed": 0.0}
    solo_its = []
    for prec in seq:
        for i, m in enumerate(ms):
            t, its = steps_time(m, member_bcs(0, m, 10), prec, max(2, args.steps // 2))
            seq[prec] += t
            if prec == "mixed":
                solo_its.append(max(its))
    value = args.batch / t_batch
    line = {"metric": "batched: simulation steps/s of independent meshes stepped as one system",
            "value": round(value, 2), "unit": "simulation-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_batch_step": round(t_batch * 1e3, 3), "higher_is_better": True,
            "meshes": args.batch, "total_tets": int(u.n_tets), "total_nodes": int(u.n_nodes),
            "tets_per_mesh": [int(m.n_tets) for m in ms], "krylov_iterations": its_b,
            "krylov_iterations_solo_max": int(max(solo_its)),
            "union_single_krylov": {"ms_per_batch_step": round(t_union * 1e3, 3), "krylov_iterations": its_u,
                                    "sim_steps_per_s": round(args.batch / t_union, 2)},
            "sequential_fp64_sim_steps_per_s": round(args.batch / seq["fp64"], 2),
            "sequential_mixed_sim_steps_per_s": round(args.batch / seq["mixed"], 2),
            "speedup_vs_sequential_fp64": round(value / (args.batch / seq["fp64"]), 3),
            "speedup_vs_sequential_mixed": round(value / (args.batch / seq["mixed"]), 3),
            "mesh_gen_s": round(tgen, 1), "dtype": "f32+f64", "data": "synthetic"}
    print(json.dumps(line), flush=True)


def oracle_step_time(n_tets, steps=1):
    """Times the FP64 oracle (C element loop + scipy assembly + aSIMPLE-FGMRES) on a cylinder of
    n_tets from rest, returns (seconds per step, T)."""
    import oracle as O

    m, _ = make_case(n_tets, seed=2)
    Q = U_PEAK * math.pi * R_CM ** 2 / 2.0
    prob = O.Problem(O.Params(rho=RHO, mu=MU, dt=DT, bdf_order=2, stab=2),
                     [O.BC(tag=0, kind="noslip"),
                      O.BC(tag=1, kind="dirichlet", time="ramp", tparams={"g0": 0.0, "g1": Q, "t0": 0.0, "tL": RAMP},
                           space="parabolic", radius=R_CM),
                      O.BC(tag=2, kind="neumann", tparams={"value": 0.0})])
    V = m.n_nodes
    uh, ph = [np.zeros((V, 3))] * 2, [np.zeros(V)] * 2
    solver = lambda A, b: O.fgmres(A, b, M=O.ASimple(A).apply, restart=40, tol=1e-8)[0]
    t0 = time.perf_counter()
    t = 0.0
    for s in range(steps):
        t += DT
        stp = O.step(m, prob, uh, ph, t, solver=solver)
        x = stp.x.reshape(-1, 4)
        uh, ph = [x[:, :3].copy(), uh[0]], [x[:, 3].copy(), ph[0]]
    return (time.perf_counter() - t0) / steps, m.n_tets


def cpu_baseline(sample_tets):
    sec, T = oracle_step_time(sample_tets, steps=1)
    # scaled to the 1M-tet workload assuming cost linear in T (optimistic for the oracle: its
    # Krylov iteration count grows with the mesh)
    value = 1.0 / (sec * 1.0e6 / T)
    return {"value": round(value, 5), "unit": "steps/s", "cores": 1, "kind": "oracle",
            "sample": f"1 BDF2 step of the oracle on a {T}-tet cylinder of the same recipe, "
                      f"{sec:.2f} s, scaled linearly to 1.0e6 tets"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O

    O.load_library()
    for _ in range(args.warmup):
        oracle_step_time(args.cpu_sample_tets, steps=1)
    secs = [oracle_step_time(args.cpu_sample_tets, steps=1) for _ in range(args.steps)]
    sec = statistics.mean(s for s, _ in secs)
    T = secs[0][1]
    value = 1.0 / (sec * 1.0e6 / T)
    line = {"impl": "reference", "metric": "time steps/s at 1M P1 tets (BDF2 VMS-LES step: assembly + aSIMPLE-GMRES)",
            "value": round(value, 5), "unit": "steps/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sec * 1e3 * 1.0e6 / T, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "poiseuille_cylinder_1M_tets (sampled)", "sample_tets": T},
            "cpu_baseline": {"value": round(value, 5), "unit": "steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} oracle steps on a {T}-tet cylinder, scaled linearly to 1e6 tets"},
            "e2e": {"value": round(value, 5), "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="both", choices=["fp64", "mixed", "both"])
    ap.add_argument("--tets", type=int, default=1_000_000)
    ap.add_argument("--cpu-sample-tets", type=int, default=40_000)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--mode", default="step", choices=["step", "serving", "batched"])
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--batch-min", type=int, default=20_000)
    ap.add_argument("--batch-max", type=int, default=300_000)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    ap.add_argument("--req-steps", type=int, default=100)
    ap.add_argument("--serve-min", type=float, default=50_000)
    ap.add_argument("--serve-max", type=float, default=400_000)
    ap.add_argument("--pool", type=int, default=4)
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--serve-budget-frac", type=float, default=0.5)
    ap.add_argument("--serve-precision", default="mixed", choices=["mixed", "fp64"])
    args = ap.parse_args()
    if args.mode == "serving":
        run_serving(args)
    elif args.mode == "batched":
        run_batched(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
