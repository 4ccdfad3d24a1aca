"""Throughput of the coupled LB/IB swimmer step (MLUPS including the IB cost)
and the HBM-roofline fraction of its dominant kernel.

Workload: the two-swimmer boxes, 256 x 128 x 128 (x = swimming axis) with two
three-bead swimmers (bead radius 6 at icosphere subdivision 3 = 642 nodes,
spacing 18, k = 0.005, Gs = 0.01, drive 1e-3, period 2000, phase pi/2),
in-line and side by side at surface gaps of 3, 5 and 8 bead radii: six boxes.
One step advances all six boxes by one coupled time step.  Synthetic inputs
(the problem has no dataset): the fluid starts at rest, the beads at their
rest shape.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

The six boxes are independent and alternate between two CUDA streams.
Under torchrun every rank runs the same six boxes on its own GPU (replicas),
timing is max over ranks and value is the whole-job aggregate; the 64-box
ensemble line partitions its boxes over the ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time


ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS incl. IBM and % of HBM roofline (FP32 vs FP16-storage vs batched) at stated error"
FALLBACK_HBM_GBS = 6800.0
E2E_CHUNK = 16  # steps between trajectory copies in the end-to-end measurement
# DRAM bytes (read + write) per launch of the main fluid kernel on one
# 256x128x128 two-swimmer box, from an ncu capture of that kernel
# (dram__bytes_read.sum + dram__bytes_write.sum, mean of both AA parities),
# for the storage formats captured (BF16 was not: reported as null).
K_LB_MAIN_DRAM_BYTES = {"f32": 560.1e6, "f16": 258.9e6}
WORKLOAD = "two_swimmer_boxes_256x128x128_x6"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=192)
    ap.add_argument("--warmup", type=int, default=16)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", dest="variants", action="store_false",
                    help="skip the FP16/BF16-storage lines")
    ap.add_argument("--no-ensemble", dest="ensemble", action="store_false",
                    help="skip the batched 64-box ensemble line")
    ap.add_argument("--ensemble-steps", type=int, default=32)
    ap.add_argument("--no-adjoint", dest="adjoint", action="store_false",
                    help="skip the adjoint (drive-gradient) line")
    ap.add_argument("--adjoint-precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--no-precision-config", dest="precision_config", action="store_false",
                    help="skip the 256^3 FP32/FP16/BF16 line")
    ap.add_argument("--precision-steps", type=int, default=64)
    ap.add_argument("--configs", action="store_true",
                    help="also measure the single-swimmer 48^3, the 256^3 precision configuration and the "
                         "paper's 1024x256x256 box (throughput, error against the oracle) and the oracle on "
                         "one core")
    return ap.parse_args()


def _boxes():
    from workloads import pair_boxes_256x128x128
    return pair_boxes_256x128x128()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def max_over_ranks(x, ws, device=None):
    """The largest x over the ranks of the default process group (x itself on
    one rank): every timing is the slowest rank's."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = device or ("cuda" if torch.cuda.is_available() else "cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _mlups(cells, steps, ms):
    """cells x steps updates in ms milliseconds, in MLUPS."""
    return cells * steps / (ms / 1e3) / 1e6


def job_mlups(ws, cells_per_step, steps, ms):
    """Whole-job throughput: each of the ws ranks advances cells_per_step cells
    per step (replicas of the same boxes), all done in ms milliseconds."""
    return ws * cells_per_step * steps / (ms / 1e3) / 1e6


def _peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """Sample SM clocks and throttle reasons with nvidia-smi during a region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not getattr(self, "out", ""):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_sample(seconds):
    """The FP64 oracle, as it stands, on one 256x128x128 two-swimmer box:
    coupled steps until `seconds` have elapsed (at least two), on every core
    of the process's affinity mask and then on one core."""
    import oracle

    def run(threads, secs):
        oracle.set_threads(threads)
        box = _boxes()[3]  # side by side, gap 3 radii
        sim = oracle.OracleSim(box)
        sim.step(1)  # first-touch of the arrays outside the timing
        n = 0
        t0 = time.perf_counter()
        while True:
            sim.step(1)
            n += 1
            dt = time.perf_counter() - t0
            if n >= 2 and dt >= secs:
                break
        return box.n_cells * n / dt / 1e6, n, dt

    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    cores = int(os.environ.get("OMP_NUM_THREADS", cores))
    mlups, n, dt = run(cores, seconds)
    one, n1, dt1 = run(1, seconds / 2)
    oracle.set_threads(cores)
    return {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{n} coupled steps of one 256x128x128 two-swimmer box (side by side, gap 3 radii), "
                      f"FP64, {dt:.1f} s",
            "single_core": {"value": one, "unit": "MLUPS", "cores": 1,
                            "sample": f"{n1} coupled steps of the same box on one core, {dt1:.1f} s"}}


def run_reference(a):
    ws, rank = _dist()
    if rank != 0:
        return
    import oracle
    box = _boxes()[3]
    sim = oracle.OracleSim(box)
    t0 = time.perf_counter()
    sim.step(1)
    t_step = time.perf_counter() - t0
    # bounded sample: the whole arm stays within about two minutes
    n_warm = max(0, min(a.warmup - 1, int(20.0 / t_step)))
    n_timed = max(2, min(a.steps, int(90.0 / t_step)))
    sim.step(n_warm)
    t0 = time.perf_counter()
    sim.step(n_timed)
    dt = time.perf_counter() - t0
    mlups = box.n_cells * n_timed / dt / 1e6
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt / n_timed * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "one of the six boxes per step (side by side, gap 3 radii)"},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"{n_timed} timed coupled steps (after {n_warm + 1} warm-up) of one "
                                       f"256x128x128 two-swimmer box, FP64; each step is one sixth of a "
                                       f"workload step"},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _run_ensemble(a, barrier, stream, ws, rank):
    """The batched-ensemble workload: 64 independent boxes (48^3, 64^3, 96^3,
    128x128x192; one or two swimmers each; seeded draws) advanced (1) box by
    box, each with its own graph-replayed steps, and (2) as one batch.  Under
    several ranks the 64 boxes are partitioned over the ranks by cell count
    (each rank steps its share; total work fixed, strong scaling) and the
    per-swimmer results are gathered to rank 0 at the end."""
    import torch
    from paper_2202_12147_gb300 import Batch, Simulation
    from paper_2202_12147_gb300.ensemble import gather_results, partition, rank_loads, swimmer_records
    from workloads import assemble, ensemble_boxes
    all_boxes = ensemble_boxes(64, seed=0)
    all_cells = [b.n_cells for b in all_boxes]
    shares = partition(all_cells, ws)
    mine = shares[rank]
    boxes = [all_boxes[i] for i in mine]
    sims = [Simulation(b.dims, assemble(b), tau=b.tau, rho0=b.rho0) for b in boxes]
    cells = sum(all_cells)  # the whole job's cells: every rank's share
    K = max(16, (a.ensemble_steps // 16) * 16)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for s in sims:
        s.lb_step(16)
    barrier()
    e0.record(stream)
    for s in sims:
        s.lb_step(K)
    e1.record(stream)
    barrier()
    seq_ms = e0.elapsed_time(e1)
    # sequential per-box launches, box after box, each step launched on its own
    K1 = max(2, K // 8)
    barrier()
    e0.record(stream)
    for s in sims:
        for _ in range(K1):
            s.lb_step(1)
    e1.record(stream)
    barrier()
    step_ms = e0.elapsed_time(e1) * K / K1
    # the same launches in round-robin order, one step of every box at a time
    barrier()
    e0.record(stream)
    for _ in range(K1):
        for s in sims:
            s.lb_step(1)
    e1.record(stream)
    barrier()
    rr_ms = e0.elapsed_time(e1) * K / K1
    batch = Batch(sims)
    tuning = batch.autotune(steps_per_trial=4)  # launch shapes timed on real steps
    batch.lb_step(16)
    barrier()
    e0.record(stream)
    batch.lb_step(K)
    e1.record(stream)
    barrier()
    bat_ms = e0.elapsed_time(e1)
    for s in sims:
        s.sync()
    batch.close()
    gathered = gather_results({i: swimmer_records(s) for i, s in zip(mine, sims)}, len(all_boxes), rank, ws)
    for s in sims:
        s.close()
    seq_ms, rr_ms, bat_ms, step_ms = (max_over_ranks(v, ws) for v in (seq_ms, rr_ms, bat_ms, step_ms))
    loads = rank_loads(all_cells, shares)
    return {"boxes": len(all_boxes), "cells": cells, "steps": K, "unit": "MLUPS", "scaling": "strong",
            "partition": {"ranks": ws, "cells_per_rank": loads, "boxes_per_rank": [len(x) for x in shares],
                          "max_over_mean": max(loads) / (sum(loads) / ws),
                          "swimmer_records_gathered": (sum(len(r) for r in gathered) if gathered is not None
                                                       else None)},
            "batched": _mlups(cells, K, bat_ms), "batched_ms_per_step": bat_ms / K,
            "sequential_launches": _mlups(cells, K, step_ms), "speedup_vs_sequential_launches": step_ms / bat_ms,
            "sequential_launches_means": "box after box, each coupled step of a box launched on its own "
                                         "(its kernels one by one, no graph)",
            "sequential": _mlups(cells, K, seq_ms), "sequential_ms_per_step": seq_ms / K,
            "speedup": seq_ms / bat_ms,
            "sequential_means": "box after box, each box replaying its own captured 16-step graphs",
            "round_robin": _mlups(cells, K, rr_ms), "speedup_vs_round_robin": rr_ms / bat_ms,
            "round_robin_means": "every step, each box launched on its own (one coupled step per call), box after box",
            "autotune": tuning}


def _run_adjoint(a, barrier, stream):
    """Gradient of a swimmer's net x displacement over one drive period with
    respect to its per-bead amplitudes and phases: one swimmer in 96^3, 1000
    steps, checkpoints every 100 steps.  Device time of the engine's forward
    and backward sweeps (CUDA events inside the library), next to the plain
    coupled step (lb_step) over the same 1000 steps."""
    import numpy as np
    import torch
    from paper_2202_12147_gb300 import Adjoint, Simulation
    from workloads import adjoint_single_96, assemble
    box = adjoint_single_96()
    asm = assemble(box)
    steps, K = 1000, 100
    eng = Adjoint(box.dims, asm, n_steps=steps, K=K, precision=a.adjoint_precision)
    eng.forward()  # warm-up sweep
    eng.backward(np.array([[1.0, 0.0, 0.0]]))
    barrier()
    d = eng.forward()
    g = eng.backward(np.array([[1.0, 0.0, 0.0]]))
    t = eng.timing()
    ws_bytes = eng.workspace_bytes
    eng.close()
    del eng
    torch.cuda.empty_cache()
    sim = Simulation(box.dims, asm, tau=box.tau, rho0=box.rho0)
    sim.lb_step(32)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.lb_step(steps)
    e1.record(stream)
    barrier()
    fwd_ms = e0.elapsed_time(e1)
    sim.sync()
    sim.close()
    return {"workload": "one swimmer (beads radius 6, 642 nodes), 96^3, one drive period of 1000 steps, "
                        "checkpoint every 100 steps", "precision": a.adjoint_precision,
            "objective": "x_cm(T) - x_cm(0)", "displacement": float(d[0, 0]),
            "gradient": {"A1": g[0, 0], "A2": g[0, 1], "A3": g[0, 2], "phi2": g[0, 4], "phi3": g[0, 5]},
            "engine_forward_ms": t["forward_ms"], "engine_backward_ms": t["backward_ms"],
            "lb_step_1000_ms": fwd_ms, "backward_over_lb_step": t["backward_ms"] / fwd_ms,
            "forward_plus_backward_over_lb_step": (t["forward_ms"] + t["backward_ms"]) / fwd_ms,
            "launches": {"forward": t["forward_launches"], "backward": t["backward_launches"]},
            "workspace_GB": ws_bytes / 1e9}


def _run_precision_256cube(a, stream, peak):
    """The precision configuration: 256^3 with two side-by-side swimmers
    (radius 6, gap 3 radii), FP32 against FP16 and BF16 storage of the
    shifted deviations (FP32 collision).  Per format: lb_step throughput over
    the timed steps (graph replays, CUDA events) and the main fluid kernel's
    bandwidth from a second run of the same steps with events around each of
    its launches.  The errors against the FP64 oracle at the stated step
    counts are checked by the long-run tests."""
    import torch
    from paper_2202_12147_gb300 import Simulation
    from workloads import assemble, pair_side_256cube
    box = pair_side_256cube()
    asm = assemble(box)
    n = max(16, (a.precision_steps // 16) * 16)
    out = {"workload": "pair_side_256cube: 256^3, two side-by-side swimmers (gap 3 radii), "
                       "inputs larger than L2", "cells": box.n_cells, "steps": n}
    for st in ("f32", "f16", "bf16"):
        sim = Simulation(box.dims, asm, tau=box.tau, rho0=box.rho0, storage=st)
        sim.lb_step(16)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.lb_step(n)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        sim.profile(True)
        sim.lb_step(n)
        lb_ms, lb_n = sim.profile_read()
        marked = sim.marked_cells()
        sim.sync()
        sim.close()
        esize = 4 if st == "f32" else 2
        bpl = (box.n_cells - marked) * 19 * 2 * esize
        ach = bpl / (lb_ms / lb_n / 1e3) / 1e9
        step_bytes = box.n_cells * 19 * 2 * esize
        out[st] = {"value": _mlups(box.n_cells, n, ms), "unit": "MLUPS", "ms_per_step": ms / n,
                   "roofline": {"kernel": "k_lb_main", "achieved": ach, "peak": peak, "frac": ach / peak,
                                "avg_launch_us": lb_ms / lb_n * 1e3, "bytes_per_launch": bpl},
                   "step_frac": step_bytes / (ms / n / 1e3) / 1e9 / peak}
    for st in ("f16", "bf16"):
        out[st]["speedup_vs_f32"] = out["f32"]["ms_per_step"] / out[st]["ms_per_step"]
    return out


def _f_dev(f, w, rho0=1.0):
    return f - w[:, None] * rho0


def _run_configs(a, stream):
    """The other configurations of the problem statement on one GPU, each with
    its error against the FP64 oracle: one swimmer in 48^3 (radius 4,
    subdivision 2, period 500) for its full 500 steps, two side-by-side
    swimmers in 256^3 (gap 3 radii) for 16 steps, and the paper's own
    1024 x 256 x 256 box with two in-line swimmers for 8 steps (the oracle's
    share of the budget); throughput of each in FP32 / FP16 / BF16 storage
    (64 / 32 timed steps for the large boxes); and the oracle's throughput on
    one core and on all."""
    import numpy as np
    import torch
    import oracle
    from paper_2202_12147_gb300 import Simulation, lattice
    from workloads import assemble, pair_side_256cube, paper_box_1024x256x256, single_swimmer_48
    cg, wg = lattice()
    co, wo = oracle.lattice()
    perm = [next(k for k in range(19) if (co[k] == cg[i]).all()) for i in range(19)]

    def u_of(f_gpu):
        fo = np.empty((f_gpu.shape[1], 19))
        fo[:, perm] = f_gpu.T
        return oracle.macros(fo)[1]

    def rel(x, y):
        return float(np.linalg.norm(x - y) / np.linalg.norm(y))

    out = {}
    for name, box, n_err, n_time in (("single_swimmer_48", single_swimmer_48(), 500, 500),
                                     ("pair_side_256cube", pair_side_256cube(), 16, 64),
                                     ("paper_box_1024x256x256", paper_box_1024x256x256(), 8, 32)):
        asm = assemble(box)
        osim = oracle.OracleSim(box, asm)
        x0 = osim.swimmer_centres()
        osim.step(n_err)
        u_ref = oracle.macros(osim.f)[1]
        d_ref = osim.swimmer_centres() - x0
        res = {"cells": box.n_cells, "error_steps": n_err, "timed_steps": n_time}
        for st in ("f32", "f16", "bf16"):
            sim = Simulation(box.dims, asm, tau=box.tau, rho0=box.rho0, storage=st)
            sim.lb_step(n_err)
            if box.n_cells > 50_000_000:  # the library's macroscopic fields (no 10 GB population copy)
                u = sim.lb_get_macros()[1].cpu().numpy().astype(np.float64)
            else:
                u = u_of(sim.get_populations())
            disp = np.array([sim.swimmer_state(k)["disp"] for k in range(sim.n_swimmers)])
            if n_err % 2:
                sim.lb_step(1)  # even parity: the timed steps replay whole graphs
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            sim.lb_step(n_time)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            sim.profile(True)  # the same steps again with the main kernel bracketed by events
            sim.lb_step(n_time)
            lb_ms, lb_n = sim.profile_read()
            marked = sim.marked_cells()
            sim.sync()
            sim.close()
            esize = 4 if st == "f32" else 2
            bw = (box.n_cells - marked) * 19 * 2 * esize / (lb_ms / lb_n / 1e3) / 1e9
            res[st] = {"MLUPS": box.n_cells * n_time / (ms / 1e3) / 1e6, "velocity_rel_l2": rel(u, u_ref),
                       # a few steps into a long drive period the swimmers have not moved yet:
                       # no relative displacement error then
                       "displacement_rel_err": (float(np.abs(disp[:, 0] - d_ref[:, 0]).max() / np.abs(d_ref[:, 0]).max())
                                                if n_err >= 0.01 * box.swimmers[0].period else None),
                       "k_lb_main_GBs": bw,
                       "timing": "MLUPS: lb_step (graph replays), CUDA events; k_lb_main_GBs: a second run of the "
                                 "same steps with events around every main-kernel launch"}
        out[name] = res
    # the oracle on one core and on all (bounded samples of the 48^3 workload)
    box = single_swimmer_48()
    all_cores = oracle.set_threads(0)
    for n_thr in (1, all_cores):
        oracle.set_threads(n_thr)
        sim = oracle.OracleSim(box)
        sim.step(1)
        t0 = time.perf_counter()
        n = 0
        while n < 2 or time.perf_counter() - t0 < 3.0:
            sim.step(1)
            n += 1
        dt = time.perf_counter() - t0
        out[f"oracle_{n_thr}_cores"] = {"MLUPS": box.n_cells * n / dt / 1e6, "steps": n, "workload": "single_swimmer_48"}
    oracle.set_threads(all_cores)
    return out


def run_ours(a):
    import torch
    import torch.distributed as dist
    from paper_2202_12147_gb300 import Simulation
    from workloads import assemble

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    boxes = _boxes()
    asms = [assemble(b) for b in boxes]
    stream = torch.cuda.current_stream()
    # the boxes are independent: they alternate between two CUDA streams, so
    # one box's immersed-boundary chain runs while another's fluid update does
    streams = [stream, torch.cuda.Stream()]

    def make(storage):
        return [Simulation(b.dims, asm, tau=b.tau, rho0=b.rho0, storage=storage, stream=streams[i % 2])
                for i, (b, asm) in enumerate(zip(boxes, asms))]

    def step_all(ss, n, e_start=None, e_stop=None):
        """n steps of every box (graph replays), both streams bracketed by
        e_start / e_stop recorded on the current stream."""
        if e_start is not None:
            e_start.record(stream)
        fork = torch.cuda.Event()
        fork.record(stream)
        streams[1].wait_event(fork)
        for x in ss:
            x.lb_step(n)
        done = torch.cuda.Event()
        done.record(streams[1])
        stream.wait_event(done)
        if e_stop is not None:
            e_stop.record(stream)

    def step_each_alone(ss, n):
        """n steps of one box after the other (for per-launch kernel times)."""
        for x in ss:
            x.lb_step(n)
            x.sync()

    sims = make(a.storage)
    N = boxes[0].n_cells

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()

    step_all(sims, a.warmup)
    for s in sims:
        s.sync()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        # timed region: the production path (lb_step, graph replays)
        barrier()
        step_all(sims, a.steps, e0, e1)
        barrier()
        ms = e0.elapsed_time(e1)
        # the same number of steps with CUDA events around every launch of
        # the main fluid kernel (the same graph schedule with event-record
        # nodes), one box at a time, for the kernel's roofline
        for s in sims:
            s.profile(True)
        step_each_alone(sims, a.steps)
        barrier()
    lb_ms, lb_n = 0.0, 0
    for s in sims:
        t, n = s.profile_read()
        lb_ms += t
        lb_n += n
        s.profile(False)
    for s in sims:
        s.sync()  # latched device errors surface here
    ms = max_over_ranks(ms, ws)
    cells_per_step = N * len(sims)
    value = job_mlups(ws, cells_per_step, a.steps, ms)
    esize = {"f32": 4, "f16": 2, "bf16": 2}[a.storage]
    # the timed kernel updates every cell outside the tiles the node stencils mark
    marked = statistics.mean(s.marked_cells() for s in sims)
    bytes_per_launch = (N - marked) * 19 * 2 * esize
    lb_avg_s = lb_ms / lb_n / 1e3
    peak, peak_kind = _peak()
    achieved = bytes_per_launch / lb_avg_s / 1e9
    launches = a.steps * len(sims) * 5  # per box-step: main fluid; prepare, gather-spread, marked fluid, interp
    step_ach = cells_per_step * 19 * 2 * esize / (ms / a.steps / 1e3) / 1e9

    variants = None
    if a.variants and a.storage == "f32":
        # the same workload with 16-bit population storage (FP32 collision)
        for s in sims:
            s.close()
        variants = {}
        for st in ("f16", "bf16"):
            vs = make(st)
            step_all(vs, a.warmup)
            barrier()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            step_all(vs, a.steps, f0, f1)
            barrier()
            vms = max_over_ranks(f0.elapsed_time(f1), ws)
            for s in vs:
                s.profile(True)
            step_each_alone(vs, a.steps)
            barrier()
            t_lb, n_lb = 0.0, 0
            for s in vs:
                t, n = s.profile_read()
                t_lb += t
                n_lb += n
                s.sync()
            vmarked = statistics.mean(s.marked_cells() for s in vs)
            vbytes = (N - vmarked) * 19 * 2 * 2
            vach = vbytes / (t_lb / n_lb / 1e3) / 1e9
            vstep = cells_per_step * 19 * 2 * 2 / (vms / a.steps / 1e3) / 1e9
            variants[st] = {"value": job_mlups(ws, cells_per_step, a.steps, vms), "unit": "MLUPS",
                            "ms_per_step": vms / a.steps, "speedup_vs_f32": ms / vms,
                            "roofline": {"achieved": vach, "peak": peak, "frac": vach / peak,
                                         "traffic": K_LB_MAIN_DRAM_BYTES.get(st),
                                         "avg_launch_us": t_lb / n_lb * 1e3, "bytes_per_launch": vbytes,
                                         "step_achieved": vstep, "step_frac": vstep / peak}}
            for s in vs:
                s.close()
        sims = []

    precision = None
    if a.precision_config and a.storage == "f32" and rank == 0:
        precision = _run_precision_256cube(a, stream, peak)

    ensemble = None
    if a.ensemble and a.storage == "f32":
        ensemble = _run_ensemble(a, barrier, stream, ws, rank)

    adjoint = None
    if a.adjoint and a.storage == "f32" and rank == 0:
        adjoint = _run_adjoint(a, torch.cuda.synchronize, stream)  # rank 0 only: no collective barrier

    e2e = None
    if not a.no_e2e:
        # End to end through the public API: structure upload from host arrays
        # (lb_init), then the steps of every box with every step's trajectory
        # points (bead centres and velocities of every swimmer) read to host.
        for s in sims:
            s.close()
        del sims
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        sims2 = make(a.storage)
        h2d = sum(asm["nodes"].nbytes * 2 + asm["tris"].nbytes * 6 for asm in asms)
        import ctypes
        from paper_2202_12147_gb300 import _lib
        # chunks of E2E_CHUNK steps (graph replays); after each chunk, one
        # asynchronous copy per box of the chunk's per-step trajectory points
        # into pinned host memory, so every step's result reaches the host
        rec = ctypes.sizeof(_lib.TrackPoint)
        n_sw = max(s.n_swimmers for s in sims2)
        host = torch.empty((len(sims2), a.steps, n_sw * rec), dtype=torch.uint8, pin_memory=True)
        d2h = 0
        done = 0
        while done < a.steps:
            k = min(E2E_CHUNK, a.steps - done)
            for s in sims2:
                s.lb_step(k)
            for b, s in enumerate(sims2):
                s.track_async(k, host[b, done:done + k])
                d2h += rec * s.n_swimmers * k
            done += k
        for s in sims2:
            s.sync()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        dt = max_over_ranks(dt, ws)
        e2e = {"value": job_mlups(ws, cells_per_step, a.steps, dt * 1e3), "unit": "MLUPS",
               "h2d_bytes_per_step": int(h2d / a.steps), "d2h_bytes_per_step": int(d2h / a.steps),
               "how": "host wall clock around lb_init of every box (structure uploaded from host arrays) and "
                      f"the steps; every step's trajectory point of every swimmer copied to pinned host memory, "
                      f"one copy per box every {E2E_CHUNK} steps"}
        for s in sims2:
            s.close()

    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        cpu = _oracle_sample(a.cpu_seconds)

    configs = None
    if a.configs and rank == 0 and ws == 1:
        configs = _run_configs(a, torch.cuda.current_stream())

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": a.storage, "data": "synthetic",
            "config": {"workload": WORKLOAD, "boxes": len(boxes), "dims": list(boxes[0].dims), "cells_per_box": N,
                       "swimmers_per_box": 2, "nodes_per_box": int(asms[0]["nodes"].shape[0]),
                       "cases": [b.name for b in boxes], "storage": f"{a.storage} shifted deviations",
                       "tau": 1.0, "delta_kernel": "peskin4", "forcing": "guo",
                       "l2": "inputs larger than L2 (populations 318 MB per box in FP32)",
                       "timing": "value: lb_step of every box over the timed steps (16-step CUDA graph replays; "
                                 "each box's step on two streams, the boxes alternating between two caller "
                                 "streams), CUDA events around both; roofline: the same number of steps right "
                                 "after, one box at a time, replaying the same 16-step graph captured with an "
                                 "event-record node before and after every main fluid-kernel launch"},
            "roofline": {"bound": "hbm", "kernel": "k_lb_main", "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": K_LB_MAIN_DRAM_BYTES.get(a.storage),
                         "bytes_per_launch": bytes_per_launch, "avg_launch_us": lb_avg_s * 1e6,
                         "launches": lb_n, "cells_per_launch": N - marked,
                         "step_achieved": step_ach, "step_frac": step_ach / peak,
                         "step_means": "every cell's 2 x 19 population values (the main and the marked-tile "
                                       "fluid updates) of every box over ms_per_step, from the timed production "
                                       "run itself"},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(),
            "variants": variants, "precision_256cube": precision, "ensemble": ensemble, "adjoint": adjoint,
        }
        if configs is not None:
            line["configs"] = configs
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
