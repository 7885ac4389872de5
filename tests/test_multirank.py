"""The multi-GPU path of bench.py on the CPU: two ranks over gloo (127.0.0.1).

bench.py runs one independent replica per GPU (the build, apply and RK4 step need no data from
another rank); the only collectives are the barriers around the timed region and the max over
ranks of the step times, which sets the whole-job throughput.  These tests check that host logic
with world_size 2 without a GPU: every rank gets the maximum, the throughput counts the nodes of
every replica, and each replica draws its own node set and field."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        step_ms = [12.5, 20.0][rank]  # the second replica is the slower one
        slowest = bench.max_over_ranks(torch, step_ms, world, "cpu")
        ns, field, C, beta, dt = bench.workload(seed_offset=rank)
        sig = [float(ns.xy[:64].sum()), float(field.value(ns.xy[:64]).sum())]
        sigs = [None] * world
        torch.distributed.all_gather_object(sigs, sig)
        out[rank] = (slowest, sigs)
    finally:
        torch.distributed.destroy_process_group()


def test_two_ranks_take_the_slowest_replica_and_draw_distinct_inputs():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    assert out[0][0] == out[1][0] == 20.0
    sig0, sig1 = out[0][1]
    assert sig0 != sig1  # each replica builds its own seeded node set and field
    # whole-job throughput: both replicas' nodes over the slowest step
    n = 512 * 512
    assert bench.replicas_throughput(world, n, 20.0) == pytest.approx(2 * n / 20e-3 / 1e6)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(torch, 7.25, 1, "cpu") == 7.25
    assert bench.replicas_throughput(1, 1000, 1.0) == pytest.approx(1.0)
    ns0, f0, *_ = bench.workload(seed_offset=0)
    ns1, f1, *_ = bench.workload(seed_offset=1)
    assert not np.array_equal(ns0.xy, ns1.xy)
