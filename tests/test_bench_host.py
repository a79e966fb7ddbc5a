"""Host-side logic of bench.py on the CPU: the multi-rank reduction of the
timed region (gloo, world size 2), the reference arm's rank-0-only rule, the
clock-sample summary and the traffic bookkeeping."""
import json
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        assert (w, r, local) == (world, rank, rank)
        bench.barrier(w)
        # rank r timed 10 + r ms and processed 100 (r + 1) units
        ms, units = bench.aggregate(10.0 + rank, 100.0 * (rank + 1), w, torch.device("cpu"))
        bench.barrier(w)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"ms": ms, "units": units}, f)
    finally:
        dist.destroy_process_group()


def test_aggregate_two_ranks_gloo(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    for r in range(world):
        got = json.loads((tmp_path / f"r{r}.json").read_text())
        # every rank sees the slowest rank's time and the sum of all units
        assert got == {"ms": 11.0, "units": 300.0}


def test_aggregate_single_rank_is_identity():
    assert bench.aggregate(3.5, 7.0, 1) == (3.5, 7.0)


def test_reference_arm_only_on_rank_zero(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = bench.parse_args(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"])
    bench.run_reference(args)
    assert capsys.readouterr().out == ""


def test_clock_summary():
    rows = ["0, 1900, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1950, 2070, 1200.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2000, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line", "0, [N/A], 2070, 1, 0, a, b, c, d"]
    s = bench.summarise_clocks(rows)
    assert s == {"sm_mhz": 1950.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert bench.summarise_clocks([]) is None


def test_traffic_bookkeeping():
    t, why = bench.sweep_traffic("4d", "mix_fp32", 1.0e9)
    if t is None:
        assert "changed" in why          # kernels edited since the capture: reported as null
    else:
        assert 0.9e9 < t < 1.1e9
    t, why = bench.sweep_traffic("2d", "fp64", 1.0e9)
    assert t is None and "no ncu capture" in why


def test_oracle_error_of_exact_and_perturbed_samples():
    """The bench line's error against the oracle: zero for the oracle's own
    values, and the planted perturbation's size otherwise (relative L2 with
    the Legendre weights, relative max), over a 2D and a 1D sample."""
    import numpy as np
    import oracle as O
    from paper_1603_07008_gb300 import workloads as W
    p = W.config2(n=16, steps=1)
    cells = np.array([0, 5, 77, 255])
    sched = O.schedule(p.grid, "strang", p.dt, p.field_list())
    exact = O.sample_after(p.grid, p.k, p.nq, p.weights, p.params, sched * 2, cells)
    e = bench.oracle_error({"steps": 2, "items": [(p, cells, exact.copy(), 6)]}, "mix_fp32")
    assert e["rel_l2"] == 0.0 and e["rel_max"] == 0.0 and e["within_bound"] and e["cells"] == 4
    bad = exact.copy()
    bad[2, 3] += 1e-3 * np.max(np.abs(exact))
    e = bench.oracle_error({"steps": 2, "items": [(p, cells, bad, 6)]}, "mix_fp32")
    assert abs(e["rel_max"] - 1e-3) < 1e-12
    w = O.l2_weights(p.k, 2)
    want = np.sqrt(np.sum((bad - exact) ** 2 * w) / np.sum(exact ** 2 * w))
    assert abs(e["rel_l2"] - want) <= 1e-15 and not e["within_bound"]
    q = W.config1()
    h = 1.0 / q.grid.n[0]
    s1 = [(0, -1, np.array([q.velocity * q.dt / h]))]
    c1 = np.array([3, 1000])
    ref = O.sample_after(q.grid, q.k, q.nq, q.weights, q.params, s1 * 100, c1)
    e = bench.oracle_error({"steps": 1, "items": [(q, c1, ref, 100)]}, "fp64")
    assert e["rel_max"] == 0.0 and e["bound"] == {"rel_max": 1e-12}
    assert bench.oracle_error(None, "mix_fp32")["note"]


def test_oracle_error_of_nodal_and_whole_state_samples():
    """The error leg's nodal cones (x-sweeps at the Gauss nodes of each
    v-cell) and its whole-state check of the self-consistent field: zero for
    the oracle's own values, the perturbation's size otherwise."""
    import numpy as np
    import oracle as O
    from paper_1603_07008_gb300 import workloads as W
    p = W.config3(n=6, steps=1)
    cells = np.array([0, 100, 1295])
    sched = O.schedule_nodal(p.grid, "strang", p.dt, p.field_list())
    exact = O.sample_after(p.grid, p.k, p.nq, p.weights, p.params, sched * 2, cells)
    e = bench.oracle_error({"steps": 2, "items": [(p, cells, exact.copy(), 12)], "nodal": True}, "mix_fp32")
    assert e["rel_max"] == 0.0 and e["within_bound"]
    plain = O.sample_after(p.grid, p.k, p.nq, p.weights, p.params,
                           O.schedule(p.grid, "strang", p.dt, p.field_list()) * 2, cells)
    e = bench.oracle_error({"steps": 2, "items": [(p, cells, plain, 12)], "nodal": True}, "fp64")
    assert e["rel_max"] > 1e-6          # the centre-velocity sweep is not the nodal one
    q = W.config2(n=16, steps=1)
    ref = O.vp_step(O.project(q.grid, q.k, q.nq, q.weights, q.params), q.grid, q.k, "strang", q.dt, 1)
    e = bench.oracle_error({"steps": 1, "whole": (q, ref.copy())}, "mix_fp32")
    assert e["rel_l2"] == 0.0 and e["cells"] == 256
    bad = ref.copy()
    bad[5, 0] += 1e-3
    assert bench.oracle_error({"steps": 1, "whole": (q, bad)}, "fp64")["rel_max"] > 0


def test_launch_counts_per_step():
    """gpu_launches counts the kernels of the timed steps: a split step builds
    each dimension's table once besides its sweeps; nodal x-sweeps build their
    node table (and, in the mixed store, the per-v-cell record) before each;
    the self-consistent field adds its two launches and builds the v-table
    after them; the 1D FP64 advection graph is one cluster launch."""
    from types import SimpleNamespace as NS

    def n(workload, storage, **info):
        return bench.launches_per_step(NS(workload=workload, storage=storage), info)

    assert n("4d", "mix_fp32", sweeps=6, ndim=4) == 10          # 6 sweeps + 4 tables
    assert n("6d", "mix_bf16", sweeps=9, ndim=6) == 15
    assert n("2d", "mix_fp32", sweeps=3, ndim=2) == 5
    assert n("batch", "mix_fp32", sweeps=3, ndim=2) == 5
    assert n("vp", "mix_fp32", sweeps=3, ndim=2) == 7           # + density and field
    # 4D nodal: 4 nodal x-sweeps (table + record + sweep), 2 v-sweeps, 2 v-tables
    assert n("4d", "mix_fp32", sweeps=6, ndim=4, nodal_x_sweeps=4) == 16
    assert n("4d", "fp64", sweeps=6, ndim=4, nodal_x_sweeps=4) == 12
    assert n("1d", "fp64", sweeps=100, ndim=1) == 1
    assert n("1d", "mix_fp32", sweeps=100, ndim=1) == 200
