"""Right-hand-side sharding across ranks on the CPU (gloo, world size 2).

The ranks run the host logic of the sharded response solve with the CPU
oracle standing in for the per-rank GPU solve; the gathered alpha must equal
a single-process solve of all frequencies."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2503_23144_gb300 import shard


def test_partition_is_balanced_and_complete():
    for n_w in (0, 1, 3, 4, 7, 64):
        for world in (1, 2, 3, 8):
            parts = [shard.partition(n_w, world, r) for r in range(world)]
            flat = [i for p in parts for i in p]
            assert flat == list(range(n_w))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.partition(4, 2, 2)


def test_gather_single_process_and_duplicate_detection():
    a = np.arange(2 * 3 * 3).reshape(2, 3, 3) + 0j
    out = shard.gather_alpha([1, 0], a, 2, 3)
    assert np.array_equal(out[1], a[0]) and np.array_equal(out[0], a[1])
    with pytest.raises(RuntimeError):
        shard.gather_alpha([0], a[:1], 2, 3)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, result_path):
    import torch.distributed as dist

    import synth
    from oracle import ccsd
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = synth.make_system(2, 5, 8, seed=3)
        model = ccsd.build(s)
        t, E, _ = ccsd.solve_ccsd(model)
        lam, _ = ccsd.solve_lambda(model, t)
        omegas = [0.0, 0.02, 0.05]

        def solve(w, c):
            return ccsd.polarizability(s, c, w, ground=(t, E, lam))

        alpha = shard.solve_sharded(solve, omegas, (0, 2), rank, world)
        if rank == 0:
            np.save(result_path, alpha)
    finally:
        dist.destroy_process_group()


def test_sharded_solve_two_gloo_ranks(tmp_path):
    import synth
    from oracle import ccsd
    out = str(tmp_path / "alpha.npy")
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    got = np.load(out)
    s = synth.make_system(2, 5, 8, seed=3)
    ref = ccsd.polarizability(s, (0, 2), [0.0, 0.02, 0.05])
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()


def _worker_fail(rank, world, port, marker):
    import datetime

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=15))
    if rank == 1:
        # this rank fails between steps: it leaves without taking part in the gather
        os._exit(3)
    try:
        shard.gather_alpha([0], np.zeros((1, 2, 2)), 2, 2)
        result = "no error"
    except Exception as e:  # the surviving rank learns of the failure instead of hanging
        result = "error: " + type(e).__name__
    with open(marker, "w") as f:
        f.write(result)
    os._exit(0)


def test_rank_failure_surfaces_as_error(tmp_path):
    marker = str(tmp_path / "rank0.txt")
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker_fail, args=(r, 2, port, marker)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert procs[1].exitcode == 3
    assert procs[0].exitcode == 0
    assert open(marker).read().startswith("error")
