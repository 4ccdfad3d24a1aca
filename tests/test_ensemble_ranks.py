"""The ensemble's distribution over ranks (one GPU per process): the
partition of the boxes by cell count and the final gather of per-swimmer
results to rank 0, on CPU with two gloo ranks; and one rank's share stepped
on the GPU against the same boxes stepped alone."""
import itertools
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_covers_every_box_once_and_is_deterministic():
    from paper_2202_12147_gb300.ensemble import partition, rank_loads
    from workloads import ensemble_boxes
    cells = [b.n_cells for b in ensemble_boxes(64, seed=0)]
    for n in (1, 2, 3, 4, 8, 64, 100):
        sh = partition(cells, n)
        assert len(sh) == n
        assert sorted(i for s in sh for i in s) == list(range(64))
        assert all(s == sorted(s) for s in sh)
        assert partition(cells, n) == sh
        loads = rank_loads(cells, sh)
        assert sum(loads) == sum(cells)
        # list scheduling bound: no rank exceeds the mean load by more than the largest box
        assert max(loads) <= sum(cells) / n + max(cells)
    with pytest.raises(ValueError):
        partition(cells, 0)


def test_partition_within_four_thirds_of_optimum_brute_force():
    """Graham's bound for longest-processing-time-first, against the optimum
    found by trying every assignment of small instances."""
    import numpy as np
    from paper_2202_12147_gb300.ensemble import partition, rank_loads
    rng = np.random.default_rng(11)
    for _ in range(30):
        m = int(rng.integers(3, 9))
        n = int(rng.integers(2, 4))
        cells = [int(v) for v in rng.choice([110592, 262144, 884736, 3145728], size=m)]
        best = min(max(sum(c for c, r in zip(cells, a) if r == k) for k in range(n))
                   for a in itertools.product(range(n), repeat=m))
        got = max(rank_loads(cells, partition(cells, n)))
        assert got <= best * 4 / 3 + 1e-9
    # a case where the greedy order matters: 3+3 on one rank, 2+2+2 on the other
    assert sorted(rank_loads([3, 3, 2, 2, 2], partition([3, 3, 2, 2, 2], 2))) == [5, 7]


def test_gather_rejects_missing_and_duplicate_boxes():
    from paper_2202_12147_gb300.ensemble import gather_results
    assert gather_results({1: "b", 0: "a"}, 2, 0, 1) == ["a", "b"]
    with pytest.raises(RuntimeError):
        gather_results({0: "a"}, 2, 0, 1)


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from paper_2202_12147_gb300.ensemble import gather_results, partition
    from workloads import ensemble_boxes
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        boxes = ensemble_boxes(64, seed=0)
        mine = partition([b.n_cells for b in boxes], ws)[rank]
        # stand-in per-box results: which rank stepped the box, and its size
        local = {i: {"rank": rank, "cells": boxes[i].n_cells, "swimmers": len(boxes[i].swimmers)} for i in mine}
        out = gather_results(local, len(boxes), rank, ws)
        q.put((rank, mine, out))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_partition_and_gather():
    import torch.multiprocessing as mp
    from paper_2202_12147_gb300.ensemble import partition, rank_loads
    from workloads import ensemble_boxes
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    boxes = ensemble_boxes(64, seed=0)
    cells = [b.n_cells for b in boxes]
    shares = partition(cells, 2)
    assert [r[1] for r in res] == shares          # both ranks computed the same partition
    assert res[1][2] is None                      # only rank 0 receives the results
    out = res[0][2]
    assert len(out) == 64
    for i, rec in enumerate(out):
        assert rec["cells"] == cells[i] and rec["swimmers"] == len(boxes[i].swimmers)
        assert i in shares[rec["rank"]]
    loads = rank_loads(cells, shares)
    assert max(loads) / min(loads) < 1.05        # the 64 boxes split evenly by cells


@pytest.mark.gpu
def test_one_rank_share_matches_boxes_stepped_alone(gpu_lib):
    """world_size 1: the share is every box, stepped as one batch; with
    deterministic spreading every box's swimmers end bitwise where the same
    box stepped alone ends."""
    from paper_2202_12147_gb300 import Simulation
    from paper_2202_12147_gb300.ensemble import EnsembleShare, swimmer_records
    from workloads import assemble, ensemble_boxes
    boxes = [b for b in ensemble_boxes(64, seed=0) if b.n_cells <= 64 ** 3][:4]
    asms = [assemble(b) for b in boxes]
    sh = EnsembleShare(boxes, asms, 0, 1, deterministic=True)
    assert sh.mine == list(range(len(boxes)))
    sh.lb_step(24)
    got = sh.gather()
    sh.close()
    for b, asm, rec in zip(boxes, asms, got):
        s = Simulation(b.dims, asm, tau=b.tau, rho0=b.rho0, deterministic=True)
        s.lb_step(24)
        assert swimmer_records(s) == rec
        s.close()
