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
FP64_PEAK_TFLOPS = 1.00            # measured DFMA probe on a GB300: 0.501 T instructions/s x 2 flops
FP32_ISSUE_PEAK_T = 35.96          # measured FP32 FMA-issue probe on a GB300, T thread-instructions/s
FP32_PEAK_TFLOPS = 2 * FP32_ISSUE_PEAK_T   # the FP32 pipe the double-float arithmetic runs on
F_STEPS = 6                        # Chebyshev steps on F per preconditioner application (library default)
# FP64-class operations of the method per tetrahedron (DFMA x 2 + DADD + DMUL executed by the FP64
# assembly kernel, counted with ncu): the algorithmic work of one element's assembly
ASM_FP64_FLOPS_PER_ELEMENT = 2948
# DRAM bytes per block of the FP32 Krylov SpMV (ncu read + write, 2,089,595-block launch)
SPMV32_DRAM_BYTES_PER_BLOCK = 71.6
# DRAM bytes per block of one staged BF16 F pass of the preconditioner (ncu read + write of one
# launch on the 817,970-tet cylinder, scaled to other sizes by the block count)
FPASS_BF16_DRAM_BYTES_PER_BLOCK = 29.8
# DRAM bytes per element of one whole persistent double-float assembly (ncu read + write of one
# launch on the 817,970-tet cylinder, scaled by the element count)
ASM_DD_PERSISTENT_DRAM_BYTES_PER_ELEMENT = 1793


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


ASSEMBLY = {}   # options.assembly when --assembly names a shape


def gpu_problem(L, m, precision, **more):
    Q = U_PEAK * math.pi * R_CM ** 2 / 2.0
    bcs = [L.BC(tag=0, kind="noslip"),
           L.BC(tag=1, kind="dirichlet", profile="parabolic", time="ramp", p=(0.0, Q, 0.0, RAMP), radius=R_CM),
           L.BC(tag=2, kind="neumann", time="constant", p=(0.0,))]
    extra = dict(smoother_bf16=1) if precision == "mixed" else {}
    extra.update(ASSEMBLY)
    extra.update(more)
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


def e2e_loop(st, u_last, p_last, t_last, dt, steps):
    """End-to-end steps through the C ABI with page-locked host buffers: returns ms per step."""
    import torch

    V = u_last.shape[0]

    def pinned(*shape):
        return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()

    hu, hp = pinned(2, V, 3), pinned(2, V)
    hu[0], hu[1] = u_last, u_last
    hp[0], hp[1] = p_last, p_last
    t_now = t_last

    def one():
        nonlocal t_now
        st.set(hu, hp, t_now)
        st.step(allow_not_converged=True)
        hu[1], hp[1] = hu[0], hp[0]
        st.get(hu[0], hp[0])
        t_now += dt

    one()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    return (time.perf_counter() - w0) * 1e3 / steps


def kernel_rooflines(stats, T, V, nnzb, prec, bf16=True):
    """Rooflines of the step's kernels from the CUDA events inside the timed steps: the assembly
    (algorithmic bytes over the measured HBM copy bandwidth, and its FP64-class flops over the pipe
    they run on), the preconditioner's F pass and the Krylov SpMV (HBM).  Returns the dominant
    kernel's roofline (most device time per step) and the table of all three."""
    peaks, src = _peaks()
    n = len(stats)
    hbm = peaks["hbm_gbs"]
    # assembly: algorithmic bytes of one step's assembly (connectivity, coordinates, history, each
    # block value written once, the right-hand side), and 2,948 FP64-class flops per element
    asm_ms = sum(s["ms_assembly_kernels"] for s in stats) / n
    n_asm = max(1, stats[0]["n_assembly_launches"])
    sv_asm = 8                                   # FP64, or the FP32 high + low parts of the dd matrix
    asm_bytes = 16 * T + V * (3 * 8 + 8 * 8) + nnzb * 16 * sv_asm + 4 * V * 8
    asm_flops = ASM_FP64_FLOPS_PER_ELEMENT * T
    dd = prec == "mixed"
    pipe = FP32_PEAK_TFLOPS if dd else FP64_PEAK_TFLOPS
    shape = {1: "assemble_color_kernel (one launch per element colour)",
             2: "assemble_chunk_kernel (one launch per chunk colour)",
             3: "assemble_chunks_persistent_kernel (one cooperative launch)"}.get(stats[0].get("assembly_mode", 0), "assembly")
    asm = {"kernel": shape + (", double-float arithmetic on the FP32 pipes" if dd else ", FP64") + "; one step's assembly",
           "bound": "alu", "achieved": round(asm_flops / (asm_ms * 1e-3) / 1e12, 4),
           "peak": pipe, "unit": "TFLOP/s (FP64-class flops of the method)",
           "frac": round(asm_flops / (asm_ms * 1e-3) / 1e12 / pipe, 4),
           "traffic": int(ASM_DD_PERSISTENT_DRAM_BYTES_PER_ELEMENT * T)
                      if dd and stats[0].get("assembly_mode", 0) == 3 else None,
           "peak_source": "measured FP32 FMA probe x 2 flops (the pipe double-float runs on)" if dd else
                          "measured FP64 FMA probe x 2 flops",
           "flops_per_element": ASM_FP64_FLOPS_PER_ELEMENT,
           "hbm_view": {"achieved_gbs": round(asm_bytes / (asm_ms * 1e-3) / 1e9, 1), "peak_gbs": hbm,
                        "frac": round(asm_bytes / (asm_ms * 1e-3) / 1e9 / hbm, 4), "algorithmic_bytes": int(asm_bytes)},
           "ms_per_step": round(asm_ms, 4), "ms_per_launch": round(asm_ms / n_asm, 4), "launches_per_step": n_asm}
    # F pass: the aSIMPLE velocity smoothing step; F sub-blocks (12 values; in the staged BF16 pass
    # the column rides in the record's padding, else 4 more bytes), the row pointers, and per node
    # the reads of d_old, r, x, diag(F)^-1 and the writes of r, d, x
    its = statistics.mean(s["iterations"] for s in stats)     # Arnoldi steps = preconditioner applications
    f_ms = statistics.median([s["ms_fpass_median"] for s in stats if s["n_fpass"] > 0] or [0.0])
    nf = F_STEPS - 1                                            # F launches per application (the first fused)
    sf = (2 if bf16 else 4) if dd else 8
    sx = 4 if dd else 8
    staged = dd and bf16
    f_bytes = nnzb * (12 * sf + (0 if staged else 4)) + 4 * (V + 1) + V * 4 * sx * 7
    fpass = None
    if f_ms > 0:
        bw = f_bytes / (f_ms * 1e-3) / 1e9
        fpass = {"kernel": ("f_step_staged_kernel (aSIMPLE velocity smoothing pass, BF16 F sub-blocks staged "
                            "into shared memory by bulk asynchronous copies)") if staged else
                           "f_step_kernel (aSIMPLE velocity smoothing pass, %s F sub-blocks)" % ("FP32" if dd else "FP64"),
                 "bound": "hbm", "achieved": round(bw, 1), "peak": hbm, "unit": "GB/s", "frac": round(bw / hbm, 4),
                 "traffic": int(FPASS_BF16_DRAM_BYTES_PER_BLOCK * nnzb) if staged and FPASS_BF16_DRAM_BYTES_PER_BLOCK else None,
                 "peak_source": src + " (burst copy)", "ms_per_launch": round(f_ms, 5),
                 "launches_per_step": round(nf * its, 1), "ms_per_step": round(f_ms * nf * its, 4),
                 "timing": "CUDA events around the plain F passes of one preconditioner application per step "
                           "(median over the steps); launches per step = (F steps - 1) x Arnoldi steps",
                 "algorithmic_bytes_per_launch": int(f_bytes)}
    # Krylov SpMV (inner FP32 in mixed precision, FP64 otherwise)
    spmv_ms = sum(s["ms_spmv"] for s in stats) / max(1, sum(s["n_spmv"] for s in stats))
    sv = 4 if dd else 8
    spmv_bytes = nnzb * (16 * sv + 4) + 4 * (V + 1) + 2 * 4 * V * sv
    spmv_bw = spmv_bytes / (spmv_ms * 1e-3) / 1e9
    spmv = {"kernel": f"spmv_kernel ({'FP32' if sv == 4 else 'FP64'} 4x4 block CSR, Arnoldi products)",
            "bound": "hbm", "achieved": round(spmv_bw, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(spmv_bw / hbm, 4),
            "traffic": int(SPMV32_DRAM_BYTES_PER_BLOCK * nnzb) if sv == 4 else None, "peak_source": src + " (burst copy)",
            "ms_per_launch": round(spmv_ms, 5), "launches_per_step": round(its, 1),
            "ms_per_step": round(spmv_ms * its, 4),
            "timing": "CUDA events around one Arnoldi SpMV launch in five (at most 4 per step); launches "
                      "per step = Arnoldi steps",
            "algorithmic_bytes_per_launch": int(spmv_bytes)}
    kernels = {"assembly": asm, "spmv": spmv}
    if fpass:
        kernels["f_pass"] = fpass
    dom = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
    roof = dict(kernels[dom])
    roof["dominant_of"] = {k: v["ms_per_step"] for k, v in kernels.items()}
    return roof, kernels


def implicit_steps(L, m, hist_u, hist_p, t_start, stream, steps):
    """The fully implicit VMS-LES step (Newton's method, each update one mixed-precision Krylov
    solve; Section 2.3's implicit u* and LES term) on the same mesh and history: one untimed step,
    then `steps` steps timed by the step's own CUDA events."""
    _, prob = gpu_problem(L, m, "mixed", implicit=1, newton_rtol=1e-8)
    st = L.State(prob, hist_u, hist_p, t_start, stream=stream)
    st.step(allow_not_converged=True)
    stats = [st.step(allow_not_converged=True) for _ in range(steps)]
    ms = statistics.mean(s["ms_total"] for s in stats)
    newton = statistics.mean(s["newton_iterations"] for s in stats)
    return {"workload": "the same cylinder and history, fully implicit (Newton) mixed precision, newton_rtol 1e-8",
            "steps_per_s": round(1e3 / ms, 3), "ms_per_step": round(ms, 3), "steps": steps,
            "newton_iterations_mean": round(newton, 2),
            "ms_per_newton_iteration": round(ms / max(newton, 1e-9), 3),
            "ms_newton_assembly_per_step": round(statistics.mean(s["ms_newton_assembly"] for s in stats), 3),
            "krylov_iterations_mean": round(statistics.mean(s["iterations"] for s in stats), 1),
            "converged": all(bool(s["converged"]) for s in stats),
            "timing": "the step's CUDA events (assembly + Newton loop), mean over the steps"}


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
    sten = args.mode == "stenosis"
    if sten:
        from synthetic import stenosis

        t0g = time.time()
        m = stenosis(R_CM, L_CM, n_tets=args.tets if args.tets != 1_000_000 else 4_000_000, seed=3 + rank)
        tgen = time.time() - t0g
        build_problem, dt_w = stenosis_problem, 5e-4
    else:
        m, tgen = make_case(args.tets, seed=2 + rank)
        build_problem, dt_w = gpu_problem, DT
    V = m.n_nodes
    stream = torch.cuda.current_stream()
    # common starting state: the FP64 path run through the warm-up steps from rest
    mesh64, prob64 = build_problem(L, m, "fp64")
    st64 = L.State(prob64, np.zeros((2, V, 3)), np.zeros((2, V)), 0.0, stream=stream)
    for _ in range(args.warmup):
        st64.step(allow_not_converged=True)
    u1, p1 = st64.get()
    # history level 1 from a second FP64 step snapshot is not kept by the API: restart BDF2 from
    # two copies of the warm state
    hist_u, hist_p, t_start = np.stack([u1, u1]), np.stack([p1, p1]), args.warmup * dt_w
    results = {}
    for prec in (["mixed", "fp64"] if args.precision == "both" else [args.precision]):
        mesh, prob = (mesh64, prob64) if prec == "fp64" else build_problem(L, m, prec)
        st = L.State(prob, hist_u, hist_p, t_start, stream=stream)
        if dist:
            dist.barrier()
        clocks = Clocks()
        clocks.start()
        ms, stats, launches = timed_steps(L, st, args.steps, 1, stream)
        clk = clocks.stop()
        _, ms = replica_throughput(ms, args.steps, dist, "cuda")
        u, p = st.get()
        results[prec] = dict(ms=ms, stats=stats, launches=launches, clocks=clk, u=u, p=p, st=st, mesh=mesh,
                             tuning=prob.assembly_tuning())
    prim = results["mixed"] if "mixed" in results else results[args.precision]
    prim_prec = "mixed" if "mixed" in results else args.precision
    info = prim["mesh"].info()
    st = prim["st"]
    amg = st.amg_levels()
    # ---- end to end through the public API, every step: the history in from page-locked host
    # buffers, the step, the solution out into the level-0 slot of the same buffers (DMA both
    # ways); the host then shifts its history levels, as a caller advancing the simulation does.
    # One untimed round first, so that the timed steps continue a consistent history.
    e2e_ms = e2e_loop(st, prim["u"], prim["p"], prim["stats"][-1]["t"], dt_w, args.steps)
    h2d, d2h = 2 * V * 4 * 8, V * 4 * 8
    # ---- per-kernel rooflines from CUDA events recorded inside the timed steps (on the state's
    # stream); the dominant kernel by device time per step is the line's roofline
    stats = prim["stats"]
    T, nnzb = info["n_tets"], info["nnz_blocks"]
    roof, kernels = kernel_rooflines(stats, T, V, nnzb, prim_prec, bf16=True)
    asm_ms = kernels["assembly"]["ms_per_step"]
    its = [s["iterations"] for s in stats]
    ms = prim["ms"]
    value = world * args.steps / (ms * 1e-3)
    line = {
        "metric": ("time steps/s at 4M P1 tets, stenosis + resistive valve (BDF2 VMS-LES step)" if sten else
                   "time steps/s at 1M P1 tets (BDF2 VMS-LES step: assembly + aSIMPLE-GMRES)"),
        "value": round(value, 3), "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prim_prec == "fp64" else "f32+f64",
        "data": "synthetic (seeded jittered-BCC Delaunay cylinder; no paper meshes available)",
        "config": {"workload": (f"stenosis_riis_womersley_{T}_tets" if sten else f"poiseuille_cylinder_{T}_tets"),
                   "n_tets": T, "n_nodes": V, "nnz_blocks": nnzb,
                   "n_colors": info["n_colors"], "precision": prim_prec, "bdf_order": 2, "dt": dt_w,
                   "gmres_rtol": 1e-8, "krylov_iterations_mean": statistics.mean(its),
                   "outer_iterations_mean": statistics.mean(s["outer_iterations"] for s in stats),
                   "schur_amg_levels": {"rows": [r for r, _ in amg], "nnz": [z for _, z in amg]},
                   "l2": "inputs larger than L2 (FP64 matrix %.0f MB > 129 MB)" % (nnzb * 16 * 8 / 1e6),
                   "mesh_gen_s": round(tgen, 1), "start": f"from rest, {args.warmup} FP64 warm-up steps"},
        "elements_per_s_assembly": round(T / (asm_ms * 1e-3), 1),
        "phase_ms": {"assembly": round(statistics.mean(s["ms_assembly"] for s in stats), 3),
                     "solve": round(statistics.mean(s["ms_solve"] for s in stats), 3)},
        "roofline": roof,
        "kernels": kernels,
        "assembly_autotuner": {"chosen": {1: "colors", 2: "chunks", 3: "persistent"}.get(prim["tuning"][0], "none"),
                               "ms_per_assembly": {k: round(v, 4) for k, v in prim["tuning"][1].items()}},
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
    if not sten and args.implicit_steps > 0:
        line["implicit"] = implicit_steps(L, m, hist_u, hist_p, t_start, stream, args.implicit_steps)
    if rank == 0 and args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_sample_tets, target_tets=T, stenosis_case=sten)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_serving(args):
    """Serving workload (continuous batching): Poisson arrivals (mean args.rate req/s) of
    simulations on cube / cylinder / stenosis geometries drawn from a pre-generated pool (sizes
    log-uniform in [args.serve_min, args.serve_max] tets), each asking for args.req_steps BDF2
    steps, admitted by a device-memory budget into the native request loop.  Reports p50/p99
    per-step latency and aggregate steps/s, beside the same requests run back to back on one
    stream (sequential FP64 GPU)."""
    import torch

    from paper_2304_12032_gb300 import build as B

    B.build()
    from paper_2304_12032_gb300 import lfx as L
    from synthetic import stenosis

    from synthetic import cube_kuhn

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rng = np.random.default_rng(5)
    # the pool: sizes log-uniform in [serve_min, serve_max], geometry kinds in turn from the three
    # single-mesh workloads (the cube of the Beltrami case, the cylinder, the stenosis)
    sizes = np.exp(rng.uniform(math.log(args.serve_min), math.log(args.serve_max), args.pool))
    pool = []
    Q = U_PEAK * math.pi * R_CM ** 2 / 2.0
    for i, nt in enumerate(sizes):
        kind = ("cube", "cylinder", "stenosis")[i % 3]
        if kind == "cube":
            nc = max(4, int(round((nt / 6.0) ** (1.0 / 3.0))))
            m = cube_kuhn(nc, length=2.0, seed=50 + i)
            bcs = [L.BC(tag=t, kind="noslip") for t in (3, 4, 5, 6)] + \
                  [L.BC(tag=1, kind="dirichlet", profile="uniform", time="ramp", p=(0.0, 10.0, 0.0, RAMP)),
                   L.BC(tag=2, kind="neumann", time="constant", p=(0.0,))]
        else:
            m = make_case(int(nt), seed=50 + i)[0] if kind == "cylinder" else stenosis(R_CM, L_CM, n_tets=int(nt), seed=50 + i)
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
            "config": {"workload": f"serving_poisson_{args.rate:g}_req_s_pool_{len(pool)}_meshes_"
                                   f"{int(args.serve_min)}_{int(args.serve_max)}_tets"},
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
        stats = [st.step(allow_not_converged=True) for _ in range(n)]
        torch.cuda.synchronize()
        wall = (time.perf_counter() - w0) / n
        its = [s["iterations"] for s in stats]
        mode, tuned = prob.assembly_tuning()
        phases = {"assembly": float(np.median([s["ms_assembly_kernels"] for s in stats])),
                  "solve": float(np.median([s["ms_solve"] for s in stats])),
                  "step_events": float(np.median([s["ms_total"] for s in stats])),
                  "wall": wall * 1e3,
                  "assembly_shape": {1: "colors", 2: "chunks", 3: "persistent"}.get(mode, "none"),
                  "autotuner_ms": {k: round(v, 3) for k, v in tuned.items()}}
        phase_log.append(phases)
        return wall, its

    u = batch(ms)
    bcs = sum((member_bcs(i, m, 10) for i, m in enumerate(ms)), [])
    phase_log = []
    t_batch, its_b = steps_time(u, bcs, "mixed", args.steps)
    batch_phases = {k: (round(v, 3) if isinstance(v, float) else v) for k, v in phase_log[0].items()}
    seq_phase = {"assembly": 0.0, "solve": 0.0}
    t_union, its_u = steps_time(u, bcs, "mixed", max(2, args.steps // 2), segmented=0)
    seq = {"fp64": 0.0, "mixed": 0.0}
    solo_its = []
    for prec in seq:
        for i, m in enumerate(ms):
            t, its = steps_time(m, member_bcs(0, m, 10), prec, max(2, args.steps // 2))
            seq[prec] += t
            if prec == "mixed":
                solo_its.append(max(its))
                seq_phase["assembly"] += phase_log[-1]["assembly"]
                seq_phase["solve"] += phase_log[-1]["solve"]
    value = args.batch / t_batch
    line = {"metric": "batched: simulation steps/s of independent meshes stepped as one system",
            "value": round(value, 2), "unit": "simulation-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_batch_step": round(t_batch * 1e3, 3), "higher_is_better": True,
            "meshes": args.batch, "total_tets": int(u.n_tets), "total_nodes": int(u.n_nodes),
            "tets_per_mesh": [int(m.n_tets) for m in ms], "krylov_iterations": its_b,
            "krylov_iterations_solo_max": int(max(solo_its)),
            "phase_ms": batch_phases,
            "sequential_mixed_phase_ms": {k: round(v, 3) for k, v in seq_phase.items()},
            "union_single_krylov": {"ms_per_batch_step": round(t_union * 1e3, 3), "krylov_iterations": its_u,
                                    "sim_steps_per_s": round(args.batch / t_union, 2)},
            "sequential_fp64_sim_steps_per_s": round(args.batch / seq["fp64"], 2),
            "sequential_mixed_sim_steps_per_s": round(args.batch / seq["mixed"], 2),
            "speedup_vs_sequential_fp64": round(value / (args.batch / seq["fp64"]), 3),
            "speedup_vs_sequential_mixed": round(value / (args.batch / seq["mixed"]), 3),
            "mesh_gen_s": round(tgen, 1), "dtype": "f32+f64", "data": "synthetic"}
    print(json.dumps(line), flush=True)


def beltrami_errors(X, tets, u, p, t):
    """Relative L2 / H1-seminorm velocity and L2 pressure (mean-free) errors against the
    Ethier-Steinman closed form at time t, with the 4-point rule (Eq. errors)."""
    from synthetic import beltrami_grad_u, beltrami_p, beltrami_u

    qa, qb = 0.5854101966249685, 0.1381966011250105
    x = X[tets]
    J = np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2)
    w = np.abs(np.linalg.det(J)) / 24.0
    Ji = np.linalg.inv(J)
    gh = np.array([[-1, -1, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    gphi = np.einsum("tmk,am->tak", Ji, gh)
    gu = np.einsum("tai,taj->tij", u[tets], gphi)
    eu = nu = eg = ng = 0.0
    ph, pe, ws = [], [], []
    for q in range(4):
        lam = np.full(4, qb)
        lam[q] = qa
        xq = np.einsum("a,tai->ti", lam, x)
        ue, ge = beltrami_u(xq, t), beltrami_grad_u(xq, t)
        uh = np.einsum("a,tai->ti", lam, u[tets])
        eu += np.sum(w * np.sum((uh - ue) ** 2, 1))
        nu += np.sum(w * np.sum(ue ** 2, 1))
        eg += np.sum(w * np.sum((gu - ge) ** 2, (1, 2)))
        ng += np.sum(w * np.sum(ge ** 2, (1, 2)))
        ph.append(np.einsum("a,ta->t", lam, p[tets]))
        pe.append(beltrami_p(xq, t))
        ws.append(w)
    ph, pe, ws = np.stack(ph), np.stack(pe), np.stack(ws)
    vol = ws.sum()
    ph, pe = ph - (ws * ph).sum() / vol, pe - (ws * pe).sum() / vol
    return (math.sqrt(eu / nu), math.sqrt(eg / ng), math.sqrt(np.sum(ws * (ph - pe) ** 2) / np.sum(ws * pe ** 2)))


def run_beltrami(args):
    """Ethier-Steinman Beltrami flow (a = pi/4, d = pi/2; closed form of Appendix A) on the unit cube,
    8^3 hexahedra split into 6 tetrahedra each (3072 tets, 729 nodes), P1-P1 VMS-LES, rho = mu = 1,
    BDF1, dt = 1e-3, 10 steps, exact (discretely flux-free) Dirichlet data on all faces, pressure
    pinned at one node: FP64 on the GPU, errors against the closed form; the FP64 oracle beside it."""
    import torch

    from paper_2304_12032_gb300 import build as B

    B.build()
    from paper_2304_12032_gb300 import lfx as L
    from synthetic import beltrami_p, beltrami_u, cube_kuhn, zero_net_flux

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n, dt, nsteps = 8, 1e-3, 10
    m = cube_kuhn(n)
    X, V = m.nodes, m.n_nodes
    bd = np.unique(m.bfaces.ravel())
    mesh = L.Mesh.from_synthetic(m)
    bcs = [L.BC(tag=t, kind="nodal") for t in range(1, 7)]
    prob = L.Problem(mesh, 1.0, 1.0, dt, 1, bcs, [], L.default_options(gmres_rtol=1e-12, gmres_max_iters=3000,
                                                                       pin_pressure_node=0))
    stream = torch.cuda.current_stream()
    data = []
    for k in range(nsteps):
        t1 = (k + 1) * dt
        ue = beltrami_u(X, t1)
        ue[bd] = zero_net_flux(X, m.bfaces, bd, ue[bd])
        data.append((ue, float(beltrami_p(X[:1], t1)[0])))

    def run(st):
        for ue, pin in data:
            for tg in range(1, 7):
                st.set_dirichlet_nodal(tg, ue)
            st.set_pressure_pin(pin)
            st.step()

    for _ in range(args.warmup):
        run(L.State(prob, beltrami_u(X, 0.0)[None], beltrami_p(X, 0.0)[None], 0.0, stream=stream))
    st = L.State(prob, beltrami_u(X, 0.0)[None], beltrami_p(X, 0.0)[None], 0.0, stream=stream)
    clocks = Clocks()
    clocks.start()
    torch.cuda.synchronize()
    n0 = L.library().lfx_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run(st)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = L.library().lfx_launch_count() - n0
    clk = clocks.stop()
    u, p = st.get()
    eu, eh, ep = beltrami_errors(X, m.tets, u, p, nsteps * dt)
    # end to end: the 10 steps with the initial history in from page-locked memory and the result out
    hu = torch.empty((1, V, 3), dtype=torch.float64, pin_memory=True).numpy()
    hp = torch.empty((1, V), dtype=torch.float64, pin_memory=True).numpy()
    ou = torch.empty((V, 3), dtype=torch.float64, pin_memory=True).numpy()
    op = torch.empty((V,), dtype=torch.float64, pin_memory=True).numpy()
    hu[0], hp[0] = beltrami_u(X, 0.0), beltrami_p(X, 0.0)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    st.set(hu, hp, 0.0)
    run(st)
    st.get(ou, op)
    e2e_s = time.perf_counter() - w0
    value = nsteps / (ms * 1e-3)
    info = mesh.info()
    line = {"metric": "time steps/s, Beltrami flow 3072 P1 tets (BDF1 VMS-LES, FP64), error vs closed form",
            "value": round(value, 2), "unit": "steps/s", "n_gpus": 1, "steps": nsteps, "warmup": args.warmup,
            "ms_per_step": round(ms / nsteps, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (structured Kuhn-split cube; closed-form data)",
            "config": {"workload": "beltrami_cube_8x8x8x6_3072_tets", "n_tets": info["n_tets"], "n_nodes": V,
                       "bdf_order": 1, "dt": dt, "gmres_rtol": 1e-12, "l2": "inputs fit in L2 (a 3072-tet problem)"},
            "errors_vs_closed_form_after_10_steps": {"u_L2": eu, "u_H1": eh, "p_L2_mean_free": ep},
            "e2e": {"value": round(nsteps / e2e_s, 2), "unit": "steps/s",
                    "h2d_bytes_per_step": int(4 * V * 8 / nsteps + 3 * V * 8), "d2h_bytes_per_step": int(4 * V * 8 / nsteps)},
            "gpu_launches": int(launches), "clocks": clk}
    if args.cpu_baseline:
        import oracle as O

        O.load_library()
        prob_o = O.Problem(O.Params(rho=1.0, mu=1.0, dt=dt, bdf_order=1, stab=2),
                           [O.BC(tag=t, kind="nodal") for t in range(1, 7)], pin_node=0)
        used = O.set_threads(os.cpu_count() or 1)
        uh, ph = [beltrami_u(X, 0.0)], [beltrami_p(X, 0.0)]
        w0 = time.perf_counter()
        for k, (ue, pin) in enumerate(data):
            stp = O.step(m, prob_o, uh, ph, (k + 1) * dt, nodal={tg: ue for tg in range(1, 7)}, pin_value=pin)
            x = stp.x.reshape(-1, 4)
            uh, ph = [x[:, :3].copy()], [x[:, 3].copy()]
        sec = (time.perf_counter() - w0) / nsteps
        O.set_threads(1)
        line["cpu_baseline"] = {"value": round(1.0 / sec, 3), "unit": "steps/s", "cores": int(used), "kind": "oracle",
                                "cpu_model": cpu_model(), "extrapolated": False,
                                "sample": f"the whole workload: {nsteps} oracle steps (direct sparse solve, element "
                                          f"loop on {used} threads)",
                                "gpu_vs_oracle_rel_l2": {"u": float(np.linalg.norm(u - uh[0]) / np.linalg.norm(uh[0])),
                                                         "p": float(np.linalg.norm((p - p.mean()) - (ph[0] - ph[0].mean())) /
                                                                    np.linalg.norm(ph[0] - ph[0].mean()))}}
    print(json.dumps(line), flush=True)


def stenosis_problem(L, m, precision):
    """The stenosis workload: cosine stenosis (75 % area reduction) in a cylinder R = 1 cm, L = 10 cm;
    Womersley inlet of flow rate Q(t) = Q_pk (1 - cos 2 pi t) / 2, Q_pk = pi R^2 33 cm/s (period 1 s,
    peak Re ~ 2000); zero traction at the outlet; a disk resistive surface (R = 1e4, eps = 0.05 cm,
    radius 0.5 cm) mid-length; blood; BDF2, dt = 5e-4 s; VMS-LES."""
    qpk = math.pi * R_CM ** 2 * 33.0
    bcs = [L.BC(tag=0, kind="noslip"),
           L.BC(tag=1, kind="dirichlet", profile="womersley", time="fourier", p=(1.0,), a=(0.5 * qpk, -0.5 * qpk),
                b=(0.0, 0.0), radius=R_CM),
           L.BC(tag=2, kind="neumann", time="constant", p=(0.0,))]
    riis = [L.RIIS(1.0e4, 0.05, (0.0, 0.0, 5.0), (0.0, 0.0, 1.0), 0.5)]
    extra = dict(smoother_bf16=1) if precision == "mixed" else {}
    extra.update(ASSEMBLY)
    opts = L.default_options(precision=precision, gmres_rtol=1e-8, **extra)
    mesh = L.Mesh.from_synthetic(m)
    return mesh, L.Problem(mesh, RHO, MU, 5e-4, 2, bcs, riis, opts)


def oracle_step_time(n_tets, steps=1, stenosis_case=False):
    """Times the FP64 oracle (C element loop + scipy assembly + aSIMPLE-FGMRES) from rest on a
    cylinder of n_tets (or the stenosis workload: Womersley inlet, resistive disk, dt = 5e-4),
    returns (seconds per step, T)."""
    import oracle as O

    dt = DT
    if stenosis_case:
        from synthetic import stenosis

        m = stenosis(R_CM, L_CM, n_tets=n_tets, seed=3)
        qpk = math.pi * R_CM ** 2 * 33.0
        dt = 5e-4
        prob = O.Problem(O.Params(rho=RHO, mu=MU, dt=dt, bdf_order=2, stab=2),
                         [O.BC(tag=0, kind="noslip"),
                          O.BC(tag=1, kind="dirichlet", time="fourier",
                               tparams={"period": 1.0, "a": [0.5 * qpk, -0.5 * qpk], "b": [0.0, 0.0]},
                               space="womersley", radius=R_CM),
                          O.BC(tag=2, kind="neumann", tparams={"value": 0.0})],
                         [O.RIIS(1.0e4, 0.05, O.disk_sdf(m.nodes, (0.0, 0.0, 5.0), (0.0, 0.0, 1.0), 0.5))])
    else:
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
        t += dt
        stp = O.step(m, prob, uh, ph, t, solver=solver)
        x = stp.x.reshape(-1, 4)
        uh, ph = [x[:, :3].copy(), uh[0]], [x[:, 3].copy(), ph[0]]
    return (time.perf_counter() - t0) / steps, m.n_tets


def cpu_model():
    """CPU model of this host (/proc/cpuinfo or lscpu), for the record."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baseline(sample_tets, steps=2, target_tets=1.0e6, stenosis_case=False):
    """The FP64 oracle (same algorithm: C element loop, scipy assembly, aSIMPLE-preconditioned
    FGMRES) on a bounded sample of the workload, single-threaded and with its element loop on every
    host core; scaled linearly in the element count to the workload (an optimistic scaling for the
    oracle, whose Krylov iteration count grows with the mesh)."""
    import oracle as O

    O.load_library()
    ncpu = os.cpu_count() or 1
    O.set_threads(1)
    sec1, T = oracle_step_time(sample_tets, steps=steps, stenosis_case=stenosis_case)
    used = O.set_threads(ncpu)
    secn, _ = oracle_step_time(sample_tets, steps=steps, stenosis_case=stenosis_case)
    O.set_threads(1)
    scale = target_tets / T
    return {"value": round(1.0 / (secn * scale), 5), "unit": "steps/s", "cores": int(used), "kind": "oracle",
            "single_core_value": round(1.0 / (sec1 * scale), 5), "cpu_model": cpu_model(), "nproc": ncpu,
            "extrapolated": True,
            "sample": f"{steps} BDF2 steps of the oracle on a {T}-tet {'stenosis' if stenosis_case else 'cylinder'} "
                      f"of the same recipe: "
                      f"{sec1:.2f} s/step on 1 core, {secn:.2f} s/step with the element loop on {used} threads; "
                      f"scaled linearly to {target_tets:.3g} tets"}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands, on the host cores, on bounded samples of
    the same workload (each timed step a sample step, scaled linearly in the element count to the
    1M-tet cylinder)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O

    O.load_library()
    ncpu = os.cpu_count() or 1
    used = O.set_threads(ncpu)
    for _ in range(args.warmup):
        oracle_step_time(args.cpu_sample_tets, steps=1)
    secs = [oracle_step_time(args.cpu_sample_tets, steps=1) for _ in range(args.steps)]
    O.set_threads(1)
    sec = statistics.mean(s for s, _ in secs)
    T = secs[0][1]
    target = 1_022_138
    value = 1.0 / (sec * target / T)
    line = {"impl": "reference", "metric": "time steps/s at 1M P1 tets (BDF2 VMS-LES step: assembly + aSIMPLE-GMRES)",
            "value": round(value, 5), "unit": "steps/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sec * 1e3 * target / T, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"poiseuille_cylinder_{target}_tets"},
            "cpu_baseline": {"value": round(value, 5), "unit": "steps/s", "cores": int(used), "kind": "oracle",
                             "cpu_model": cpu_model(), "extrapolated": True,
                             "sample": f"{args.steps} oracle steps on a {T}-tet cylinder of the same recipe (element "
                                       f"loop on {used} threads), scaled linearly to {target} tets", "sample_tets": T},
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
    ap.add_argument("--cpu-sample-tets", type=int, default=100_000)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--assembly", default="auto", choices=["auto", "colors", "chunks", "persistent"],
                    help="assembly launch shape (auto: the library's autotuner picks)")
    ap.add_argument("--implicit-steps", type=int, default=3,
                    help="fully implicit (Newton) steps timed after the semi-implicit ones (0: none)")
    ap.add_argument("--mode", default="step", choices=["step", "stenosis", "beltrami", "serving", "batched"])
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--batch-min", type=int, default=20_000)
    ap.add_argument("--batch-max", type=int, default=300_000)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    ap.add_argument("--req-steps", type=int, default=100)
    ap.add_argument("--serve-min", type=float, default=50_000)
    ap.add_argument("--serve-max", type=float, default=2_000_000)
    ap.add_argument("--pool", type=int, default=24)
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--serve-budget-frac", type=float, default=0.5)
    ap.add_argument("--serve-precision", default="mixed", choices=["mixed", "fp64"])
    args = ap.parse_args()
    if args.assembly != "auto":
        ASSEMBLY["assembly"] = args.assembly
    if args.mode == "serving":
        run_serving(args)
    elif args.mode == "beltrami" and args.impl != "reference":
        run_beltrami(args)
    elif args.mode == "batched":
        run_batched(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
