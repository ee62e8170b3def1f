"""Host-side tests of bench.py: two gloo ranks on the CPU run the same
barrier / max-over-ranks / aggregation helpers that the GPU replicas use with
NCCL (replicas share nothing else); the clock record's parsing."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    w, r, local, pg = bench.dist_setup(world, backend="gloo")
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(pg)
    t_rank = 0.5 + rank          # rank 1 is the slowest
    t_max = bench.allreduce_max(pg, t_rank)
    units = bench.allreduce_sum(pg, 100.0 * (rank + 1))   # ranks process 100 and 200 units
    srcs, scaling = bench.rank_sources(list(range(5)), "each", w, rank)
    out[rank] = (t_max, bench.aggregate_rate(units, t_max), srcs, scaling)
    bench.barrier(pg)
    dist.destroy_process_group()


def test_two_rank_max_time_and_aggregate():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        t_max, rate, srcs, scaling = out[r]
        assert t_max == 1.5
        assert rate == pytest.approx(300.0 / 1.5)
        assert scaling == "strong"
    assert out[0][2] + out[1][2] == list(range(5))   # the sources are split, each solved once


def test_single_process_defaults(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    import bench
    w, r, local, pg = bench.dist_setup(1)
    assert (w, r, pg) == (1, 0, None)
    assert bench.allreduce_max(pg, 3.0) == 3.0
    assert bench.aggregate_rate(10.0, 2.0) == 5.0
    assert bench.rank_sources([1, 2, 3], "batch", 1, 0) == ([1, 2, 3], "weak")
    assert bench.rank_sources([7], "one", 4, 3) == ([7], "weak")   # one source: every replica solves it


def test_clock_summary_parses_samples_and_reasons():
    """The clock record attached to every bench line: median SM clock under
    load, the maximum, and every throttle reason seen Active at least once
    (nvidia-smi csv, noheader, nounits)."""
    import bench
    cs = bench.ClockSampler(0)
    cs.lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 950.3, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 950.3, 0x0, Not Active, Not Active, Not Active, Not Active",   # unreadable sample
        "garbage",
    ]
    s = cs.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    cs.lines = ["0, 1500, 2070, 700, 0x48, Active, Not Active, Active, Not Active"]
    assert cs.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    cs.lines = []
    assert cs.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_named_workloads_and_l2_note():
    """Each named bench workload builds with its stated grid and batch; the
    numeric aliases name the same workloads; the L2 note matches the sizes."""
    import bench
    for name, (n, nrhs, nsrc) in {"homogeneous_48": (48, 1, 1), "gaussian_lens_288": (288, 1, 1),
                                  "layered_inclusion_224x16": (224, 16, 16)}.items():
        w, sources, k, how, desc = bench.resolve_workload(name)
        assert (w.n, k, len(sources)) == (n, nrhs, nsrc) and desc
        assert name.startswith(w.name)
    gen, how, desc = bench.WORKLOADS["geophysical_960x4"]
    assert (gen, how) == ("geophysical", "each")
    assert set(bench.CONFIG_ALIAS.values()) == set(bench.WORKLOADS)
    assert bench.l2_note(289 ** 3, 1).startswith("inputs larger than L2 (each fine complex64 field set 193 MB")
    assert bench.l2_note(49 ** 3, 1).startswith("inputs smaller than L2")


def test_reference_arm_line(tmp_path):
    """bench.py --impl reference (the oracle on the host cores) prints one JSON
    line with the contract's keys, for the workload selected by name or alias."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--config", "1"], capture_output=True, text=True, timeout=600,
                         env=dict(os.environ, RANK="0"))
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ["metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"]:
        assert k in line, k
    assert line["impl"] == "reference" and line["config"]["workload"] == "homogeneous_48"
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_workload_names_used_by_the_tests_exist():
    """Every workload the full-size GPU tests and the bench name resolves in
    hz_workloads, to the generator of that medium at its default size."""
    import re
    import bench
    import hz_workloads as W
    here = os.path.dirname(os.path.abspath(__file__))
    names = set()
    for f in os.listdir(here):
        if f.endswith(".py"):
            src = open(os.path.join(here, f)).read()
            names |= set(re.findall(r'by_name\("(\w+)"\)', src))
            names |= set(re.findall(r'\("(\w+_\d+(?:x\d+)?)", \d+\)', src))
    assert {"gaussian_lens_288", "geophysical_960x4", "layered_inclusion_224x16", "random_field_152x8"} <= names
    assert names <= set(W.WORKLOADS) and set(bench.WORKLOADS) <= set(W.WORKLOADS)
    for name in ("homogeneous_48", "random_field_152x8"):
        w = W.by_name(name)
        assert name.startswith(w.name) and w.n == int(re.search(r"_(\d+)", name).group(1))


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs the oracle and prints; the other ranks
    exit 0 at once without output."""
    import subprocess
    import sys
    import time
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    t0 = time.perf_counter()
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2"],
                         capture_output=True, text=True, timeout=300,
                         env=dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1"))
    assert out.returncode == 0 and out.stdout.strip() == ""
    assert time.perf_counter() - t0 < 60


def test_partition_covers_each_source_once():
    from paper_2608_22946_gb300 import replicas
    for n in (1, 4, 7, 16):
        for world in range(1, n + 1):
            parts = [replicas.partition(n, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1


def _grad_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group(backend="gloo")
    import hz_workloads as W
    from oracle import gradient as og
    from paper_2608_22946_gb300 import replicas
    w = W.random_field(n=20, n_pml=4, nsrc=4, nrec_side=3)
    d_obs = og.synthetic_data(w.c_true, w.n_pml, w.h, w.omega, w.sources, w.receivers)

    def misfit_grad(src, d):
        J, g, _ = og.misfit_and_gradient(w.c, w.n_pml, w.h, w.omega, src, w.receivers, d)
        return J, torch.from_numpy(g)

    J, g = replicas.sharded_misfit_gradient(misfit_grad, w.sources, d_obs, world, rank)
    out[rank] = (J, g.numpy())
    dist.destroy_process_group()


def test_two_ranks_split_the_sources_and_sum_the_gradient(monkeypatch):
    """Replica gradient: each of two gloo ranks evaluates the adjoint-state
    misfit and gradient for half of the sources (the oracle stands in for the
    per-rank solver here); one all-reduce gives every rank the misfit and the
    gradient of all sources, equal to the single-process evaluation."""
    import numpy as np
    import hz_workloads as W
    from oracle import gradient as og
    # one BLAS thread per rank (the spawned ranks inherit it): a multithreaded
    # BLAS in two spawned processes beside torch's own threads stalls here
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        monkeypatch.setenv(var, "1")
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_grad_worker, args=(world, port, out), nprocs=world, join=True)
    w = W.random_field(n=20, n_pml=4, nsrc=4, nrec_side=3)
    d_obs = og.synthetic_data(w.c_true, w.n_pml, w.h, w.omega, w.sources, w.receivers)
    J_ref, g_ref, _ = og.misfit_and_gradient(w.c, w.n_pml, w.h, w.omega, w.sources, w.receivers, d_obs)
    for r in range(world):
        J, g = out[r]
        assert J == pytest.approx(J_ref, rel=1e-12)
        assert np.allclose(g, g_ref, rtol=1e-12, atol=1e-12 * np.abs(g_ref).max())
