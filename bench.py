#!/usr/bin/env python
"""Benchmark: three-grid preconditioned FGMRES solve of the IOFD Helmholtz
system on one GB300 (or N replicas), plus the stencil roofline.

Workload (default): Gaussian lens, 256^3 interior + 16-point PML (288^3
intervals, 289^3 = 24.1 M fine nodes), ppw 6 at the minimum velocity, one
centre source, complex64 hierarchy with FP64 outer Krylov scalars and FP64
iterative refinement to relative residual 1e-6.

One step = one helmholtz_solve call (b = Q f, FGMRES + Algorithm 1 with FP64
refinement, u = Q v) on the resident model.  The headline value is the
fine-grid update rate N_h * nrhs * PC_calls / t_step (one update = one fine
node through one outer FGMRES step with its three-grid preconditioner call),
summed over ranks.  Replicas (N > 1) solve independent copies: no collective
on the data path ("scaling": "weak").

Other workloads: --workload homogeneous_48 | layered_inclusion_224x16 (16
sources batched); --stencil-only times the fine-grid A_h apply alone.

--impl reference times the CPU oracle (the plain complex128 implementation
of the paper's method) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fine-grid stencil GUpdates/s (%HBM peak); time-to-solution at rel res 1e-6 vs FP64"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


# Workloads by name: hz_workloads generator, how its sources are solved
# ("one": the first source only; "batch": all sources as one batch of
# right-hand sides; "each": every source in turn, one right-hand side in flight),
# and the "data" description of the JSON line.  The numeric aliases 1-3 and 5
# of --config name the same workloads.
WORKLOADS = {
    "gaussian_lens_288": ("gaussian_lens", "one", "seeded Gaussian-lens velocity, point source"),
    "homogeneous_48": ("homogeneous", "one", "constant velocity, centre point source"),
    "layered_inclusion_224x16": ("layered_inclusion", "batch",
                                 "seeded five-layer medium with a fast sphere, 16 point sources"),
    "geophysical_960x4": ("geophysical", "each",
                          "seeded depth gradient with a salt-like body and 3% noise, 4 point sources"),
}
CONFIG_ALIAS = {"1": "homogeneous_48", "2": "gaussian_lens_288", "3": "layered_inclusion_224x16",
                "5": "geophysical_960x4"}
L2_BYTES = 129e6


def resolve_workload(name):
    """(workload, sources solved per step, right-hand sides in flight, how the
    sources are solved, data description) of a named workload."""
    import hz_workloads as W
    gen, how, desc = WORKLOADS[name]
    w = getattr(W, gen)()
    sources = list(w.sources[:1]) if how == "one" else list(w.sources)
    nrhs = len(sources) if how == "batch" else 1
    return w, sources, nrhs, how, desc


def l2_note(n_nodes, nrhs):
    """How the timed inputs relate to the 129 MB L2 (the step is not re-flushed)."""
    mb = 8.0 * n_nodes * nrhs / 1e6
    if 8.0 * n_nodes * nrhs > L2_BYTES:
        return f"inputs larger than L2 (each fine complex64 field set {mb:.0f} MB)"
    return f"inputs smaller than L2 ({mb:.1f} MB per fine complex64 field set): L2-resident timing"


_T0 = time.perf_counter()


def log(msg):
    print(f"[bench {time.perf_counter() - _T0:8.1f}s] {msg}", file=sys.stderr, flush=True)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    def __init__(self, dev):
        self.dev = dev
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + CLOCK_Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(gpus, backend=None):
    """One process per GPU (torchrun sets RANK / LOCAL_RANK / WORLD_SIZE).  Replicas
    exchange only the step time (max over ranks) and a barrier around the timed
    region; NCCL on GPUs, gloo when asked (host-side tests)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend=backend or os.environ.get("HZ_DIST_BACKEND", "nccl"))
        pg = dist
    return world, rank, local, pg


def _on_gpu(pg):
    return pg is not None and pg.get_backend() == "nccl"


def barrier(pg, dev=None):
    if pg is not None:
        if _on_gpu(pg) and dev is not None:
            pg.barrier(device_ids=[dev])
        else:
            pg.barrier()


def allreduce_max(pg, x):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if _on_gpu(pg) else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(pg, x):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if _on_gpu(pg) else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def aggregate_rate(units_all_ranks, t_max):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return units_all_ranks / t_max


def rank_sources(sources, how, world, rank):
    """The sources this rank solves: a multi-source workload is split across
    the ranks (strong scaling of a fixed source list); a one-source workload is
    solved by every rank (weak scaling, independent replicas)."""
    from paper_2608_22946_gb300 import replicas
    if how == "one" or world == 1:
        return list(sources), "weak"
    a, b = replicas.partition(len(sources), world, rank)
    return list(sources[a:b]), "strong"


# ----------------------------------------------------------------------------
# oracle (CPU) timing: the reference arm and the cpu_baseline leg
# ----------------------------------------------------------------------------
ORACLE_SAMPLE_N = 48


def oracle_sample(workload_name):
    """Full oracle solve (FGMRES + Algorithm 1, complex128) of the same medium
    recipe on a 48^3 grid (8-point PML, ppw 6) to 1e-6; returns the update
    rate in GUpdates/s, seconds and a description."""
    import numpy as np
    import hz_workloads as W
    from oracle import iofd
    from oracle import threegrid as tg
    if workload_name == "gaussian_lens":
        w = W.gaussian_lens(n=ORACLE_SAMPLE_N, n_pml=8)
    elif workload_name == "layered_inclusion":
        w = W.layered_inclusion(n=ORACLE_SAMPLE_N, n_pml=8, nsrc=1)
    else:
        w = W.homogeneous(n=ORACLE_SAMPLE_N, n_pml=8)
    t0 = time.perf_counter()
    prob = iofd.make_problem(w.c, w.n_pml, w.h, w.omega, w.gamma_max)
    Q = iofd.operator_Q(prob)
    b = Q(iofd.point_sources(prob, w.sources[:1])[0])
    v, info = tg.solve(prob, b, tg.Params(tol=1e-6))
    dt = time.perf_counter() - t0
    N = w.N
    value = N * info.pc_calls / dt / 1e9
    threads = os.environ.get("OMP_NUM_THREADS") or os.environ.get("OPENBLAS_NUM_THREADS")
    cores = int(threads) if threads else (os.cpu_count() or 1)
    desc = (f"oracle (numpy complex128) full solve to 1e-6 of the {w.name} recipe at {w.n}^3 "
            f"({N} nodes, {info.pc_calls} PC calls, {dt:.1f} s); rate = N*PC/t")
    return value, dt, cores, desc


def run_reference(args):
    # the oracle runs on the host of rank 0 only; other ranks exit at once
    if int(os.environ.get("RANK", "0")) != 0:
        return
    gen = WORKLOADS[args.workload][0]
    for _ in range(args.warmup):
        oracle_sample(gen)
    vals = []
    t_all = time.perf_counter()
    for _ in range(max(1, args.steps)):
        v, dt, cores, desc = oracle_sample(gen)
        vals.append((v, dt))
    t_all = time.perf_counter() - t_all
    value = statistics.median([v for v, _ in vals])
    ms = 1000.0 * statistics.median([d for _, d in vals])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GUpdates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": args.workload, "sample": f"{gen}_{ORACLE_SAMPLE_N}"},
            "cpu_baseline": {"value": value, "unit": "GUpdates/s", "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "GUpdates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def solve_step(s, sources, how, v, u, noconv):
    """One step: every source of this rank solved (a batch at once, or one
    right-hand side at a time into the same buffers).  Returns the summed
    preconditioner calls and the last stats."""
    pc, st = 0, None
    groups = [sources] if how != "each" else [[src] for src in sources]
    for g in groups:
        _, _, st = s.helmholtz_solve(g, v_out=v, u_out=u, allow_noconv=noconv)
        pc += st["pc_calls"]
    return pc, st


def time_apply(s, hz, level, op, nrhs, stream, K=20, mode="apply"):
    """Average duration of one fine-grid operator application (apply, or the
    two-sweep Jacobi map of the fine smoother) on the launching stream, K
    launches after 3 warm-ups; inputs larger than L2."""
    import torch
    x = torch.randn((nrhs,) + s.level_shape[level], dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    if mode == "jacobi":
        f = lambda: s.iofd_jacobi(x, level=level, nsweeps=2, out=y, stream=stream)
    else:
        f = lambda: s.iofd_apply(x, op=op, level=level, out=y, stream=stream)
    for _ in range(3):
        f()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(K):
        f()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1000.0 / K


def run_gpu(args):
    import numpy as np
    import torch

    import paper_2608_22946_gb300 as hz

    world, rank, local, pg = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    w, all_sources, nrhs, how, data_desc = resolve_workload(args.workload)
    sources, scaling = rank_sources(all_sources, how, world, rank)
    if how == "batch":
        nrhs = len(sources)
    params = hz.default_params(tol=1e-6, precision=hz.HZ_C64, block=1 if args.block else 0)
    noconv = False
    if args.max_pc:
        # profiling runs: cap the preconditioner calls (same kernel mix, bounded length)
        params.max_pc = args.max_pc
        noconv = True
    c_host = torch.from_numpy(np.ascontiguousarray(w.c, dtype=np.float64).reshape(-1)).pin_memory()
    c_dev = c_host.to("cuda", non_blocking=True)
    log(f"workload {w.name} n={w.n} ready; rank {rank} solves {len(sources)} source(s), {nrhs} in flight")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = hz.Solver(w.n, w.n_pml, w.h, w.omega, c_dev, params=params, max_nrhs=nrhs)
    torch.cuda.synchronize()
    t_create_cold = time.perf_counter() - t0   # includes the z-block autotuner (first create in this process)
    del c_dev
    torch.cuda.empty_cache()
    N = w.N
    v = torch.empty((nrhs,) + s.shape, dtype=torch.complex128, device="cuda")
    u = torch.empty_like(v)
    for it in range(args.warmup):
        pc, st = solve_step(s, sources, how, v, u, noconv)
        log(f"warmup {it}: pc={pc} passes={st['refine_passes']} rel={st['rel_res']:.2e} t={st['t_solve']:.3f}s")
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    barrier(pg, dev)
    torch.cuda.synchronize()
    l0 = hz.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    pcs, stats = [], []
    with ClockSampler(dev) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            pc, st = solve_step(s, sources, how, v, u, noconv)
            pcs.append(pc)
            stats.append(st)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(pg, dev)
    launches = hz.kernel_launches() - l0
    t_step = ev0.elapsed_time(ev1) / 1000.0 / args.steps
    log(f"timed: {1000 * t_step:.1f} ms per step, pc per step {pcs}")
    t_max = allreduce_max(pg, t_step)
    pc = pcs[-1]
    units = allreduce_sum(pg, float(N * (nrhs if how == "batch" else 1) * pc))
    rel = max(st["rel_res"] for st in stats)
    value = aggregate_rate(units, t_max) / 1e9
    n_src_all = allreduce_sum(pg, float(len(sources))) if world > 1 else len(sources)

    result = {"metric": METRIC, "value": value, "unit": "GUpdates/s", "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": 1000.0 * t_max, "higher_is_better": True,
              "scaling": scaling, "vs_baseline": None, "dtype": "c64",
              "value_kind": ("solver fine-grid update rate: fine nodes x right-hand sides x preconditioner calls "
                             "per second of solve (one update = one fine node through one outer FGMRES step with "
                             "its three-grid preconditioner call); the stencil's own rate is "
                             "stencil_gupdates_per_s"),
              "data": f"synthetic ({data_desc})",
              "config": {"workload": args.workload,
                         "grid_intervals": w.n, "n_pml": w.n_pml, "fine_nodes": N, "sources": int(n_src_all),
                         "rhs_in_flight": nrhs, "ppw": 6, "tol": 1e-6,
                         "precision": "c64 hierarchy, FP64 outer scalars + refinement",
                         "krylov": "block FGMRES over the right-hand sides in flight" if args.block
                                   else "independent FGMRES per right-hand side (batched kernels)",
                         "parallelism": (f"replicas x{world}, sources split across ranks" if scaling == "strong"
                                         else f"replicas x{world}"),
                         "l2": l2_note(N, nrhs)},
              "time_to_solution_s": t_max, "pc_calls": pc, "rel_res": rel,
              "refine_passes": stats[-1]["refine_passes"], "t_setup_s": stats[-1]["t_setup"],
              "device_gib": stats[-1]["device_bytes"] / 2 ** 30,
              "zblock_tuned": {"rectangle": stats[-1].get("zblock"), "frame": stats[-1].get("zblock_frame")},
              "gpu_launches": int(launches), "clocks": clk.summary()}

    if rank == 0:
        pk, pk_kind = peaks()
        # --- roofline of the dominant kernels: the fine-grid complex64 stencil
        # (A_h apply, 20 B/node) and the fine-grid two-sweep Jacobi map (the
        # smoother of S_h; 8 (g) + 8 (1/diag) + 4 (kappa) + 8 (y) = 28 B/node)
        del u
        torch.cuda.empty_cache()
        t_k = time_apply(s, hz, 0, hz.HZ_OP_A, nrhs, stream)
        achieved = 20 * N * nrhs / t_k / 1e9
        traffic = None
        tf = os.path.join(ROOT, "profiles", "stencil_traffic.json")
        if os.path.exists(tf) and args.workload == "gaussian_lens_288":
            with open(tf) as f:
                traffic = json.load(f).get("bytes_per_launch_fine_288")
        log(f"stencil apply {1000 * t_k:.3f} ms")
        result["stencil_gupdates_per_s"] = N * nrhs / t_k / 1e9
        if nrhs > 1:
            # the same apply with one right-hand side: the batched kernels share each
            # row's coefficient evaluation between right-hand sides
            t_1 = time_apply(s, hz, 0, hz.HZ_OP_A, 1, stream)
            result["stencil_single_rhs_gupdates_per_s"] = N / t_1 / 1e9
            result["stencil_batched_over_single"] = (N * nrhs / t_k) / (N / t_1)
        result["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                              "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
                              "kernel": "k_fwd_rect + k_fwd_frame (A_h, complex64, fine grid, one application)",
                              "peak_kind": pk_kind, "gupdates_per_s": N * nrhs / t_k / 1e9,
                              "avg_launch_ms": 1000 * t_k, "bytes_per_node": 20}
        t_j = time_apply(s, hz, 0, None, nrhs, stream, mode="jacobi")
        ach_j = 28 * N * nrhs / t_j / 1e9
        result["roofline_smoother"] = {"bound": "hbm", "achieved": ach_j, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                       "frac": ach_j / pk["hbm_gbs"], "traffic": None,
                                       "kernel": "k_fwd_rect + k_fwd_frame, two-sweep Jacobi map J_2(A_h) "
                                                 "(complex64, fine grid)",
                                       "peak_kind": pk_kind, "gupdates_per_s": N * nrhs / t_j / 1e9,
                                       "avg_launch_ms": 1000 * t_j, "bytes_per_node": 28}
        log(f"jacobi map {1000 * t_j:.3f} ms")
        # --- accuracy against a converged FP64 solution and the plain FP64 GPU solve
        if not args.no_fp64 and how != "each":
            result["fp64_solve"] = fp64_leg(hz, w, sources[:1], v[:1], t_max / (nrhs if how == "batch" else 1),
                                            params)
        # --- end to end through the public API with host buffers
        u_host = torch.empty((nrhs,) + s.shape, dtype=torch.complex128).pin_memory()
        u2 = torch.empty_like(v)
        # a second handle beside the resident one must fit (the 961^3 workload
        # holds 213 GiB): otherwise release the resident handle first
        free_b, _ = torch.cuda.mem_get_info()
        if hz.workspace_bytes(w.n, w.n_pml, w.h, w.omega, params=params, max_nrhs=nrhs) > 0.9 * free_b:
            s.close()
            torch.cuda.empty_cache()
        e2e_t = []
        src_bytes = len(sources) * (3 * 4 + 2 * 8)
        for it in range(1 + args.e2e_steps if args.e2e_steps > 0 else 0):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cd = c_host.to("cuda", non_blocking=True)
            se = hz.Solver(w.n, w.n_pml, w.h, w.omega, cd, params=params, max_nrhs=nrhs)
            del cd
            pce, st = solve_step(se, sources, how, v, u2, noconv)
            u_host.copy_(u2, non_blocking=True)
            torch.cuda.synchronize()
            se.close()
            if it >= 1:
                e2e_t.append(time.perf_counter() - t0)
        te = statistics.median(e2e_t) if e2e_t else float("nan")
        log(f"e2e {e2e_t}")
        result["e2e"] = None if not e2e_t else {
            "value": N * (nrhs if how == "batch" else 1) * pce / te / 1e9, "unit": "GUpdates/s",
            "h2d_bytes_per_step": int(c_host.numel() * 8 + src_bytes),
            "d2h_bytes_per_step": int(u_host.numel() * 16), "time_to_solution_s": te,
            "includes": "H2D velocity, hz_create (set-up; z-blocks from this process's tuning cache), solve, "
                        "D2H of u, hz_destroy",
            "first_create_s": t_create_cold,
            "first_create_note": "the first hz_create of the process, including the z-block autotuner that "
                                 "later creates for the same sizes skip; add it once to e2e for a cold start"}
        # --- CPU oracle baseline (bounded sample)
        if not args.no_cpu:
            cv, cdt, cores, desc = oracle_sample(w.name)
            log(f"oracle sample {cdt:.1f}s")
            result["cpu_baseline"] = {"value": cv, "unit": "GUpdates/s", "cores": cores, "kind": "oracle",
                                      "sample": desc}
        result["context"] = ("paper: 18.1 s on 64 A100 for ~340 wavelengths/direction (2048^3, tol 1e-4); "
                             "not comparable hardware or workload")
        print(json.dumps(result), flush=True)
    s.close()
    if pg is not None:
        pg.destroy_process_group()


def fp64_leg(hz, w, sources, v_mixed, t_mixed, params):
    """The mixed-precision solution against a complex128 GPU solve converged to
    1e-10 (the reference), the plain complex128 GPU solve to the same 1e-6
    tolerance (time, calls), and the mixed solve at the tightened tolerance
    that brings its error against the reference to 1e-6 or below."""
    import torch
    out = {}
    p64 = hz.default_params(tol=1e-10, precision=hz.HZ_C128, max_pc=4000)
    s64 = hz.Solver(w.n, w.n_pml, w.h, w.omega, w.c, params=p64, max_nrhs=1)
    ref = torch.empty((1,) + s64.shape, dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, st_ref = s64.helmholtz_solve(sources, v_out=ref, want_u=False)
    torch.cuda.synchronize()
    t_ref = time.perf_counter() - t0
    nref = torch.linalg.vector_norm(ref[0])
    err = lambda x: float(torch.linalg.vector_norm(x[0] - ref[0]) / nref)
    out["reference"] = {"precision": "c128 throughout", "tol": 1e-10, "rel_res": st_ref["rel_res"],
                        "pc_calls": st_ref["pc_calls"], "time_s": t_ref}
    log(f"fp64 reference {t_ref:.2f}s pc={st_ref['pc_calls']} rel={st_ref['rel_res']:.2e}")
    # the plain FP64 GPU solve at the benchmark tolerance
    s64.set_params(hz.default_params(tol=1e-6, precision=hz.HZ_C128))
    v64 = torch.empty_like(ref)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, st64 = s64.helmholtz_solve(sources, v_out=v64, want_u=False)
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t0
    out.update({"time_to_solution_s": t64, "pc_calls": st64["pc_calls"], "rel_res": st64["rel_res"],
                "fp64_vs_reference_rel_l2": err(v64), "mixed_vs_reference_rel_l2": err(v_mixed),
                "speedup_mixed_over_fp64": t64 / t_mixed, "tol": 1e-6})
    s64.close()
    del v64
    # the mixed solve tightened until its error against the reference is <= 1e-6
    sm = hz.Solver(w.n, w.n_pml, w.h, w.omega, w.c, params=params, max_nrhs=1)
    vm = torch.empty_like(ref)
    for tol in (1e-7, 1e-8, 1e-9):
        sm.set_params(hz.default_params(tol=tol, precision=hz.HZ_C64))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, stm = sm.helmholtz_solve(sources, v_out=vm, want_u=False)
        torch.cuda.synchronize()
        tm = time.perf_counter() - t0
        e = err(vm)
        out.setdefault("mixed_tightened", []).append({"tol": tol, "time_s": tm, "pc_calls": stm["pc_calls"],
                                                      "rel_res": stm["rel_res"], "vs_reference_rel_l2": e})
        if e <= 1e-6:
            out["mixed_at_1e-6_error"] = {"tol": tol, "time_s": tm, "vs_reference_rel_l2": e,
                                          "speedup_over_fp64_at_1e-6": t64 / tm}
            break
    sm.close()
    return out


def run_stencil_only(args):
    """Time one complex64 operator application alone (default: the fine-grid
    A_h apply the roofline line reports; --level / --op select another level
    and operator), K launches after 3 warm-ups.  --no-autotune keeps the fixed
    z-block heuristic (fewer launches before the timed ones, for profilers)."""
    import torch
    import paper_2608_22946_gb300 as hz
    w, _, _, _, _ = resolve_workload(args.workload)
    params = hz.default_params(autotune=0 if args.no_autotune else 1)
    s = hz.Solver(w.n, w.n_pml, w.h, w.omega, w.c, params=params, max_nrhs=1)
    L, op = args.level, getattr(hz, "HZ_OP_" + args.op)
    x = torch.randn((1,) + s.level_shape[L], dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        s.iofd_apply(x, op=op, level=L, out=y, stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        s.iofd_apply(x, op=op, level=L, out=y, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1000.0 / args.steps
    pk, _ = peaks()
    NL = x[0].numel()
    gbs = 20 * NL / t / 1e9
    print(json.dumps({"kernel": f"forward stencil {args.op} complex64, level {L}", "workload": w.name, "n": w.n,
                      "nodes": NL, "ms": 1000 * t, "gupdates_per_s": NL / t / 1e9, "gb_per_s": gbs,
                      "frac_hbm": gbs / pk["hbm_gbs"]}), flush=True)
    s.close()


# The paper's one-A100 results on its benchmark media (Table 5; complex single
# precision, 512^3 intervals with 8 PML layers, ppw 6, FGMRES(5) to 1e-4):
# preconditioner calls, solve time in s, solve time per call in s.
PAPER_A100_512 = {"homogeneous": (19, 5.512, 0.290), "lens": (12, 4.545, 0.379),
                  "wedge": (29, 10.863, 0.375), "barrier": (32, 11.970, 0.374)}


def run_paper_media(args):
    """The paper's single-GPU benchmark media at its settings (tol 1e-4,
    complex64 hierarchy; one FP64 true residual confirms the result), one JSON
    line per medium and tolerance, with the paper's one-A100 figures beside ours
    (different hardware: context, not a ratio target).  --tols and --precision
    re-run its tolerance and precision studies (Tables 2 and 3)."""
    import torch
    import hz_workloads as W
    import paper_2608_22946_gb300 as hz
    media = args.media.split(",") if args.media else list(W.PAPER_MEDIA)
    tols = [float(t) for t in args.tols.split(",")]
    prec = hz.HZ_C128 if args.precision == "c128" else hz.HZ_C64
    for kind, tol in [(k, t) for k in media for t in tols]:
        w = W.paper_medium(kind, n=args.mesh)
        params = hz.default_params(tol=tol, precision=prec, refine=0 if args.paper_protocol else 1)
        c_dev = torch.from_numpy(w.c).to("cuda", torch.float64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = hz.Solver(w.n, w.n_pml, w.h, w.omega, c_dev, params=params, max_nrhs=1)
        torch.cuda.synchronize()
        t_create = time.perf_counter() - t0
        del c_dev
        sts = []
        for it in range(args.warmup + args.steps):
            _, _, st = s.helmholtz_solve(w.sources)
            if it >= args.warmup:
                sts.append(st)
        t_solve = statistics.median(st["t_solve"] for st in sts)
        st = sts[-1]
        pc = st["pc_calls"]
        row = {"medium": kind, "mesh": w.n, "n_pml": w.n_pml, "nodes": w.N, "tol": tol,
               "pc_calls": pc, "refine_passes": st["refine_passes"], "rel_res": st["rel_res"],
               "t_setup_s": st["t_setup"], "t_create_s": t_create, "t_solve_s": t_solve,
               "solve_per_pc_s": t_solve / max(pc, 1), "device_gib": st["device_bytes"] / 2 ** 30,
               "zblock": [st["zblock"], st["zblock_frame"]],
               "precision": ("c128 throughout" if prec == hz.HZ_C128 else
                             ("c64 throughout, stopped by its c64 true residual (the paper's protocol)"
                              if args.paper_protocol else "c64 hierarchy + FP64 residual")),
               "data": "synthetic (the paper's medium formula, centre source)"}
        if w.n == 512 and kind in PAPER_A100_512 and tol == 1e-4 and prec == hz.HZ_C64:
            p_pc, p_t, p_tpc = PAPER_A100_512[kind]
            row["paper_1xA100"] = {"pc_calls": p_pc, "t_solve_s": p_t, "solve_per_pc_s": p_tpc,
                                   "source": "Table 5"}
        print(json.dumps(row), flush=True)
        s.close()
        del s
        torch.cuda.empty_cache()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gaussian_lens_288", choices=sorted(WORKLOADS))
    ap.add_argument("--config", default=None, choices=sorted(CONFIG_ALIAS), help=argparse.SUPPRESS)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--block", action="store_true",
                    help="block FGMRES over the right-hand sides in flight (multi-source workloads)")
    ap.add_argument("--stencil-only", action="store_true")
    ap.add_argument("--level", type=int, default=0, help="--stencil-only: grid level (0 = h, 1 = 2h, 2 = 4h)")
    ap.add_argument("--op", default="A", choices=["A", "B", "Q"], help="--stencil-only: operator")
    ap.add_argument("--no-autotune", action="store_true", help="--stencil-only: fixed z-block heuristic")
    ap.add_argument("--max-pc", type=int, default=0, help="profiling only: cap preconditioner calls")
    ap.add_argument("--paper-media", action="store_true",
                    help="the paper's benchmark media (homogeneous, lens, wedge, barrier) at tol 1e-4")
    ap.add_argument("--media", default="", help="comma-separated subset for --paper-media")
    ap.add_argument("--mesh", type=int, default=512, help="intervals per direction for --paper-media")
    ap.add_argument("--tols", default="1e-4", help="comma-separated tolerances for --paper-media")
    ap.add_argument("--precision", default="c64", choices=["c64", "c128"], help="for --paper-media")
    ap.add_argument("--paper-protocol", action="store_true",
                    help="for --paper-media: one complex64 FGMRES solve to tol (no FP64 refinement), as the paper")
    args = ap.parse_args()
    if args.config:
        args.workload = CONFIG_ALIAS[args.config]
    if args.paper_media:
        run_paper_media(args)
    elif args.stencil_only:
        run_stencil_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
