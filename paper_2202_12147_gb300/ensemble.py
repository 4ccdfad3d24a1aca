"""An ensemble of independent periodic boxes spread over ranks, one GPU per
process (torch.distributed: NCCL between GPUs, gloo on CPU).

Every box is its own problem (Sec. 2: a periodic box with its swimmers), so
the boxes exchange nothing while they step.  Each rank takes a share of the
boxes balanced by cell count (the fluid update, which moves a fixed number of
bytes per cell, is nearly all of a step's cost), advances its share as one
batch (lb_batch_*: one set of launches per step for all its boxes), and the
per-swimmer observables are gathered to rank 0 at the end, in the
ensemble's box order.  The gather is the only collective.
"""
from __future__ import annotations


def partition(cells, n_ranks):
    """Balance boxes of the given cell counts over n_ranks ranks.

    Longest processing time first: the boxes in order of decreasing cell
    count (equal counts by index) each go to the rank with the fewest cells
    so far (equal loads: the lowest rank).  The largest load is at most 4/3
    of the optimum (Graham 1969).  Returns one ascending list of box indices
    per rank; every box appears exactly once.  Deterministic, so every rank
    computes the same partition without communicating."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(cells)), key=lambda i: (-int(cells[i]), i))
    load = [0] * n_ranks
    share = [[] for _ in range(n_ranks)]
    for i in order:
        r = min(range(n_ranks), key=lambda k: (load[k], k))
        share[r].append(i)
        load[r] += int(cells[i])
    return [sorted(s) for s in share]


def rank_loads(cells, shares):
    """Cells held by each rank under a partition."""
    return [sum(int(cells[i]) for i in s) for s in shares]


def swimmer_records(sim):
    """The observables of every swimmer of one box (Sec. 3: centre of mass
    x_cm, displacement, mean velocity over the last completed drive period)
    as plain Python values, ready to gather."""
    out = []
    for s in range(sim.n_swimmers):
        st = sim.swimmer_state(s)
        out.append({"step": int(st["step"]), "x_cm": [float(v) for v in st["x_cm"]],
                    "disp": [float(v) for v in st["disp"]], "periods": int(st["periods"]),
                    "v_period": [float(v) for v in st["v_period"]], "re_swim": float(st["re_swim"])})
    return out


def gather_results(local, n_boxes, rank, world_size, dst=0):
    """Collect {box index: result} from every rank on rank dst, as a list in
    box order (None on the other ranks).  With one rank no collective runs.
    Raises if a box is missing or reported twice."""
    if world_size > 1:
        import torch.distributed as dist
        parts = [None] * world_size if rank == dst else None
        dist.gather_object(dict(local), parts, dst=dst)
    else:
        parts = [dict(local)]
    if rank != dst:
        return None
    merged = {}
    for p in parts:
        for k, v in p.items():
            if k in merged:
                raise RuntimeError(f"box {k} reported by two ranks")
            merged[k] = v
    missing = [k for k in range(n_boxes) if k not in merged]
    if missing:
        raise RuntimeError(f"boxes {missing} were not reported")
    return [merged[k] for k in range(n_boxes)]


class EnsembleShare:
    """This rank's share of an ensemble: its boxes' simulations (each with its
    own caller-owned buffers on this rank's GPU) stepped as one batch.

    boxes: box descriptions with dims, n_cells, tau, rho0, forcing, kernel
    and g; structures: the host structure of each box (nodes, triangles,
    beads, swimmers; the format Simulation takes), one per box."""

    def __init__(self, boxes, structures, rank, world_size, storage="f32", deterministic=False):
        from .sim import Batch, Simulation
        if len(structures) != len(boxes):
            raise ValueError("one structure per box")
        self.n_boxes = len(boxes)
        self.shares = partition([b.n_cells for b in boxes], world_size)
        self.mine = self.shares[rank]
        self.rank, self.world_size = rank, world_size
        self.cells = sum(boxes[i].n_cells for i in self.mine)
        self.sims = []
        for i in self.mine:
            b = boxes[i]
            self.sims.append(Simulation(b.dims, structures[i], tau=b.tau, rho0=b.rho0, forcing=b.forcing,
                                        kernel=b.kernel, g=b.g, storage=storage, deterministic=deterministic))
        self.batch = Batch(self.sims) if self.sims else None

    def lb_step(self, n=1):
        if self.batch is not None:
            self.batch.lb_step(n)

    def autotune(self, steps_per_trial=4):
        return self.batch.autotune(steps_per_trial) if self.batch is not None else None

    def results(self):
        """{box index: per-swimmer records} of this rank's boxes (synchronises)."""
        return {i: swimmer_records(s) for i, s in zip(self.mine, self.sims)}

    def gather(self, dst=0):
        return gather_results(self.results(), self.n_boxes, self.rank, self.world_size, dst)

    def close(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        for s in self.sims:
            s.close()
        self.sims = []
