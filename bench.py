"""Benchmark: block-sparse GEMM GFLOP/s and seconds per LNV step on the 4096-atom Si SZP cell,
FP64 products and split-BF16 tensor-core products.

A step is one Li-Nunes-Vanderbilt step (cq_lnv_step): two trial evaluations (5 block
products each), the update, the electron-number corrections (3 products each) and the full
evaluation at the new point (7 products), plus traces, gradients and the line search.
Inputs: diamond Si, 8x8x8 conventional cells (4096 atoms, a = 10.26 bohr, seeded 0.1 bohr
jitter), 9 orbitals per atom (36,864 orbitals), S and H from the two-centre model cut at
14 bohr, L on a 16-bohr pattern started by Palser-Manolopoulos after Hotelling inversion of
S.  Patterns, task lists, the inverse and the start are built before the timed region.

The FP64 leg (value, e2e, roofline) times K steps after W warm-up steps; the split leg
restarts from the same L and times K split-BF16 steps, and reports the energy and L
differences between the two trajectories; the emulated-FP64 leg does the same with digit-
plane products.  The converge leg (N = 1) times the target criterion: seconds until the
energy stays within 1e-6 Ha/atom of the FP64 solution, plain FP64 LNV from the
Palser-Manolopoulos start against the learned start with split-BF16 steps and FP64
refinement.  Prints one JSON line (rank 0).  Under torchrun
(N > 1) every rank solves its own replica of the cell ("replicas only": the path has no
exchange step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = {"workload": "Si diamond 4096 atoms SZP (9 orb/atom, 36864 orbitals)",
            "ncell": 8, "a_bohr": 10.26, "sigma_bohr": 0.1, "seed": 2, "r_S": 14.0,
            "r_L": 16.0, "r_X": 30.0, "r_U": 44.0, "n_electrons": 16384}
BF16_FALLBACK_TFLOPS = 1900.0
# DRAM bytes per launch of the FP64 product kernel over the launches of one LNV step of the
# 4096-atom cell, from one ncu capture of the current kernel
# (profiles/bsmm_f64_traffic_si4096.md)
FP64_TRAFFIC_PER_LAUNCH = 90.66e9
# The same for the split-BF16 and the emulated-FP64 tile kernels (one ncu pass over one LNV
# step of each leg; profiles/bsmm_split_ncu_si1728.md, profiles/bsmm_emu_ncu_si1728.md)
SPLIT_TRAFFIC_PER_LAUNCH = 157.85e9
EMU_TRAFFIC_PER_LAUNCH = 374.46e9
TRAFFIC_SOURCE = "ncu dram bytes per launch, one LNV step of this cell"


METRIC = ("block-sparse GEMM GFLOP/s (useful FP64 flops) & s per LNV step, Si SZP; "
          "FP64 (value) and split-BF16 (split)")


class Replicas:
    """N independent replicas, one per rank (the path has no exchange step): a barrier that
    also drains the device, the maximum of a per-rank time, and the sum of per-rank work.
    `dist` is torch.distributed with an initialised group, or None for one process."""

    def __init__(self, dist, device):
        self.dist, self.device = dist, device

    def barrier(self):
        import torch
        if self.device.type == "cuda":
            torch.cuda.synchronize(self.device)
        if self.dist is not None:
            self.dist.barrier()

    def _reduce(self, x, op):
        if self.dist is None:
            return float(x)
        import torch
        tt = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(tt, op=op)
        return float(tt.item())

    def max(self, x):
        return self._reduce(x, self.dist.ReduceOp.MAX if self.dist else None)

    def sum(self, x):
        return self._reduce(x, self.dist.ReduceOp.SUM if self.dist else None)

    def rate(self, units, ms):
        """Whole-job throughput: the units all ranks processed over the slowest rank's time
        (ms), in units per second."""
        return self.sum(units) / (self.max(ms) * 1e-3)


def workload_name(n_atoms):
    return f"Si diamond {n_atoms} atoms SZP (9 orb/atom, {9 * n_atoms} orbitals)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cq", choices=["cq", "reference"])
    ap.add_argument("--ncell", type=int, default=8, help="cells per edge (8 = 4096 atoms)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-split", action="store_true")
    ap.add_argument("--only-split", action="store_true",
                    help="skip the FP64 leg (profiling the tensor-core path)")
    ap.add_argument("--hotelling-steps", type=int, default=12)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-emu", action="store_true",
                    help="skip the emulated-FP64 (digit planes on tensor cores) leg")
    ap.add_argument("--no-converge", action="store_true",
                    help="skip the convergence leg (learned start + split-BF16 + FP64 against "
                         "plain FP64, to within 1e-6 Ha/atom)")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the split-vs-oracle check on the 512-atom SZP cell")
    ap.add_argument("--sweep", default=None,
                    help="comma-separated cells per edge (e.g. 4,6,8,10,12): seconds per LNV step "
                         "against atom count (linear scaling), split-BF16 at every size, FP64 "
                         "up to --sweep-fp64-max cells per edge")
    ap.add_argument("--sweep-fp64-max", type=int, default=8)
    ap.add_argument("--apply-only", action="store_true",
                    help="with --converge: only the learned start and its split-BF16 phase on "
                         "the cell (no plain FP64 solve, no FP64 refinement), for cells whose "
                         "FP64 solve is too long for the bench")
    ap.add_argument("--solvers", action="store_true",
                    help="the solver options on the cell: Hotelling against the least-squares "
                         "(CG) overlap inverse, and plain against T-preconditioned FP64 LNV to "
                         "RMS gradient 1e-8 (steps and seconds)")
    ap.add_argument("--train-cells", type=int, default=6,
                    help="with --converge: training cells for the learned start")
    ap.add_argument("--train-ncell", type=int, default=3,
                    help="with --converge: cells per edge of a training cell (3: 216 atoms)")
    ap.add_argument("--train-split", action="store_true",
                    help="with --converge: solve the training cells with split-BF16 steps")
    ap.add_argument("--converge", action="store_true",
                    help="time full minimisations (plain FP64 vs learned guess + split-BF16 + "
                         "FP64 refinement) instead of the step benchmark")
    ap.add_argument("--products", default=None,
                    help="comma-separated product types of an LNV step to time one by one on "
                         "the cell with seeded random operands instead of the step benchmark: "
                         "X (L.S -> P_X), U (S.X -> P_U), R (U.X -> P_L); one untimed product, "
                         "then --steps timed ones (for kernel profiling)")
    ap.add_argument("--converge-emu", action="store_true",
                    help="the cell minimised to RMS gradient 1e-8 with FP64 products and with "
                         "emulated-FP64 tensor-core products only, from the same start")
    ap.add_argument("--batch-c4", action="store_true",
                    help="the batched workload at its full shape (32 cells of 500-8000 atoms, "
                         "mixed 5/9/13-orbital species) in sub-batches, split-BF16 LNV steps")
    ap.add_argument("--c4-atoms", type=int, default=9000,
                    help="with --batch-c4: atoms per sub-batch at most")
    ap.add_argument("--prec", default="split", choices=["fp64", "split", "emu"],
                    help="with --products: the product's precision")
    return ap.parse_args()


BATCH_CELLS = [((3, 3, 3), 0.05, 14.0), ((4, 3, 3), 0.03, 16.0), ((4, 4, 3), 0.06, 12.0),
               ((4, 4, 4), 0.045, 15.0)]


def run_batch(args, dev, rep):
    """Batched heterogeneous cells (reduced form of the 32-cell workload): four cells of
    216-512 atoms, densities 0.03-0.06 atoms/A^3, species mixed from 5/9/13 orbitals,
    r_L 12-16 bohr (r_S = r_L - 2), solved as one batch: one launch per product for all
    cells, per-cell scalars, LNV phases replayed as CUDA graphs, FP64 lane splits autotuned."""
    import torch

    from paper_2205_08941_gb300 import cq
    from paper_2205_08941_gb300 import inputs as I
    cells, Ss, Hs = [], [], []
    for k, (shape, dens, rl) in enumerate(BATCH_CELLS):
        cell = I.mixed_cell(shape, dens, 0.1, 3 + k)
        S, H = I.overlap_hamiltonian_species(cell, I.silicon_model(rl - 2.0))
        cells.append(cell)
        Ss.append(S)
        Hs.append(H)
    pos, nb, start, boxes = I.concat_cells(cells)
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    ctx = cq.Context(dev, stream=stream)
    ctx.set_autotune(True)
    t = lambda a, dt: torch.tensor(a, dtype=dt, device=f"cuda:{dev}")
    rS = [c[2] - 2.0 for c in BATCH_CELLS]
    rL = [c[2] for c in BATCH_CELLS]
    pS = ctx.pattern_batch(t(pos, torch.float64), start, boxes, t(nb, torch.int32), rS)
    pL = ctx.pattern_batch(t(pos, torch.float64), start, boxes, t(nb, torch.int32), rL)

    def up(pairs_list):
        i = np.concatenate([pb.i + start[k] for k, pb in enumerate(pairs_list)]).astype(np.int32)
        j = np.concatenate([pb.j + start[k] for k, pb in enumerate(pairs_list)]).astype(np.int32)
        sizes = np.concatenate([np.diff(pb.off) for pb in pairs_list])
        off = np.zeros(sizes.shape[0] + 1, dtype=np.int64)
        np.cumsum(sizes, out=off[1:])
        v = np.concatenate([pb.values for pb in pairs_list])
        return ctx.scatter(pS, t(i, torch.int32), t(j, torch.int32), t(off, torch.int64),
                           t(v, torch.float64))

    S, H = up(Ss), up(Hs)
    T = ctx.zeros(pL)
    torch.cuda.synchronize()
    ctx.hotelling_init(pS, S, pL, T)
    for _ in range(10):
        ctx.hotelling_step(pS, S, pL, T)
    n_occ = [2.0 * c.n_atoms for c in cells]
    L = ctx.zeros(pL)
    torch.cuda.synchronize()
    ctx.pm_guess_cells(pS, S, H, pL, T, pL, L, n_occ)
    L_start = L.clone()
    steps = 2

    def timed_steps(graphs, prec=cq.CQ_FP64):
        """`steps` timed steps from the PM start, after four untimed ones (a graph phase runs
        eagerly on its first use and is captured on its second, so the untimed steps let the
        phases the timed steps use be captured first)."""
        L.copy_(L_start)
        ctx.set_graphs(graphs)
        lnv = ctx.lnv_cells(pS, S, H, pL, L, [2 * x for x in n_occ], prec=prec)
        for _ in range(4):
            lnv.step()
        n0 = cq.kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e0.record(stream)
        reps = [lnv.step() for _ in range(steps)]
        e1.record(stream)
        stream.synchronize()
        return lnv, reps, e0.elapsed_time(e1), cq.kernel_launches() - n0

    # the same steps with eager launches, for the launch gaps the graphs remove
    lnv_e, _, ms_eager, _ = timed_steps(False)
    lnv_e.close()
    lnv, reps, ms_graph, launches = timed_steps(True)
    ms = rep.max(ms_graph)
    flops = rep.sum(sum(r[0]["flops"] for r in reps))  # r[0]: the batch total, on every cell
    out = {"workload": "4 cells, " + ", ".join(f"{c.n_atoms} atoms" for c in cells)
                       + "; species 5/9/13 orbitals mixed per atom; reduced from 32 cells",
           "value": flops / (ms * 1e-3) / 1e9, "unit": "GFLOP/s", "dtype": "f64",
           "ms_per_step": ms / steps, "graphs": True, "autotune": True,
           "ms_per_step_eager_launches": ms_eager / steps,
           "gpu_launches": int(launches),
           "energy_per_atom": [r["energy"] / c.n_atoms for r, c in zip(reps[-1], cells)],
           "gnorm": [r["gnorm"] for r in reps[-1]]}
    lnv.close()
    # the same steps with split-BF16 products on the mixed bases (graphs on)
    lnv_s, reps_s, ms_s, launches_s = timed_steps(True, cq.CQ_SPLIT_BF16X3)
    ms_s = rep.max(ms_s)
    flops_s = rep.sum(sum(r[0]["flops"] for r in reps_s))
    out["split"] = {"value": flops_s / (ms_s * 1e-3) / 1e9, "unit": "GFLOP/s",
                    "dtype": "bf16x3 split, fp32 accumulate, fp64 traces",
                    "ms_per_step": ms_s / steps, "speedup_vs_fp64_step": ms / ms_s,
                    "gpu_launches": int(launches_s),
                    "energy_diff_per_atom_vs_fp64": [
                        abs(a["energy"] - b["energy"]) / c.n_atoms
                        for a, b, c in zip(reps_s[-1], reps[-1], cells)]}
    lnv_s.close()
    ctx.close()
    return out


def c4_cells(n=32, seed0=3):
    """The batched workload's cells: cell k from seed seed0 + k -- atoms uniform in
    [500, 8000] (diamond lattices of 8 nx ny nz atoms near that count), density uniform in
    0.03-0.06 atoms/A^3, r_L uniform in 12-16 bohr (r_S = r_L - 2), species 5/9/13 per atom."""
    from paper_2205_08941_gb300 import inputs as I
    out = []
    for k in range(n):
        rng = np.random.default_rng(seed0 + k)
        target = rng.uniform(500, 8000)
        dens = rng.uniform(0.03, 0.06)
        rl = rng.uniform(12.0, 16.0)
        m = target / 8.0
        nz = max(1, int(np.floor(m ** (1.0 / 3.0))))
        ny = max(1, int(round(np.sqrt(m / nz))))
        nx = max(1, int(round(m / (ny * nz))))
        out.append((I.mixed_cell((nx, ny, nz), dens, 0.1, seed0 + k), dens, rl))
    return out


def _c4_inputs(k):
    """Cell k of the batched workload with its S and H pair blocks (host only, no CUDA; run
    in a spawned worker)."""
    from paper_2205_08941_gb300 import inputs as I
    cell, dens, rl = c4_cells()[k]
    S, H = I.overlap_hamiltonian_species(cell, I.silicon_model(rl - 2.0))
    return cell, dens, rl, S, H


def run_batch_c4(args, dev):
    """The batched workload at its full shape, split-BF16 LNV steps: the 32 cells of
    c4_cells in sub-batches of consecutive cells of at most --c4-atoms atoms (one batch of
    cells fits in HBM; the whole workload would need about 1.5 TB of FP64 matrices); per
    sub-batch the patterns, a 10-step Hotelling inverse and the PM start (untimed), then two
    untimed and two timed LNV steps of all its cells, LNV phases replayed as CUDA graphs.
    The first sub-batch is also timed with FP64 products.  Reports the seconds of one LNV
    step of all 32 cells (the sum over sub-batches) and the useful GFLOP/s."""
    import torch

    from paper_2205_08941_gb300 import build as B
    B.build()
    from paper_2205_08941_gb300 import cq
    from paper_2205_08941_gb300 import inputs as I
    import concurrent.futures as cf
    import multiprocessing as mp
    t0 = time.perf_counter()
    cells = c4_cells()
    # S and H of the cells built by spawned host workers ahead of the GPU work
    pool = cf.ProcessPoolExecutor(max_workers=max(1, min(16, (os.cpu_count() or 2) - 1)),
                                  mp_context=mp.get_context("spawn"))
    futures = [pool.submit(_c4_inputs, k) for k in range(len(cells))]
    torch.cuda.set_device(dev)
    t = lambda a, dt: torch.tensor(a, dtype=dt, device=f"cuda:{dev}")
    subs, cur, n_cur = [], [], 0
    for k, c in enumerate(cells):
        if cur and n_cur + c[0].n_atoms > args.c4_atoms:
            subs.append(cur)
            cur, n_cur = [], 0
        cur.append(k)
        n_cur += c[0].n_atoms
    subs.append(cur)
    rows, t_gen = [], 0.0
    for q, ks in enumerate(subs):
        tg = time.perf_counter()
        got = [futures[k].result() for k in ks]
        t_gen += time.perf_counter() - tg  # time the GPU waited for inputs
        sub = [(x[0], x[1], x[2]) for x in got]
        SH = [(x[3], x[4]) for x in got]
        del got
        cl = [c[0] for c in sub]
        pos, nb, start, boxes = I.concat_cells(cl)
        stream = torch.cuda.Stream(dev)
        torch.cuda.synchronize()
        ctx = cq.Context(dev, stream=stream)
        pS = ctx.pattern_batch(t(pos, torch.float64), start, boxes, t(nb, torch.int32),
                               [c[2] - 2.0 for c in sub])
        pL = ctx.pattern_batch(t(pos, torch.float64), start, boxes, t(nb, torch.int32),
                               [c[2] for c in sub])

        def up(pairs_list):
            i = np.concatenate([pb.i + start[k] for k, pb in enumerate(pairs_list)]).astype(np.int32)
            j = np.concatenate([pb.j + start[k] for k, pb in enumerate(pairs_list)]).astype(np.int32)
            sizes = np.concatenate([np.diff(pb.off) for pb in pairs_list])
            off = np.zeros(sizes.shape[0] + 1, dtype=np.int64)
            np.cumsum(sizes, out=off[1:])
            v = np.concatenate([pb.values for pb in pairs_list])
            return ctx.scatter(pS, t(i, torch.int32), t(j, torch.int32), t(off, torch.int64),
                               t(v, torch.float64))

        S, H = up([x[0] for x in SH]), up([x[1] for x in SH])
        del SH
        T = ctx.zeros(pL)
        ctx.hotelling_init(pS, S, pL, T)
        for _ in range(10):
            ctx.hotelling_step(pS, S, pL, T)
        n_occ = [2.0 * c.n_atoms for c in cl]
        L = ctx.zeros(pL)
        ctx.pm_guess_cells(pS, S, H, pL, T, pL, L, n_occ)
        del T
        ctx.release_cache()  # the set-up's FP64 task lists: the split steps need none
        L0 = L.clone()
        row = {"cells": len(sub), "atoms": int(sum(c.n_atoms for c in cl)),
               "orbitals": int(sum(int(c.nb.sum()) for c in cl))}
        precs = [("split", cq.CQ_SPLIT_BF16X3)] + ([("fp64", cq.CQ_FP64)] if q == 0 else [])
        for name, prec in precs:
            L.copy_(L0)
            ctx.set_graphs(True)
            lnv = ctx.lnv_cells(pS, S, H, pL, L, [2 * x for x in n_occ], prec=prec)
            for _ in range(2):
                lnv.step()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            stream.synchronize()
            e0.record(stream)
            reps = [lnv.step() for _ in range(2)]
            e1.record(stream)
            stream.synchronize()
            ms = e0.elapsed_time(e1) / 2
            flops = sum(r[0]["flops"] for r in reps) / 2
            row[name] = {"s_per_step": ms / 1e3, "gflops": flops / (ms * 1e-3) / 1e9,
                         "energy_per_atom": [r["energy"] / c.n_atoms
                                             for r, c in zip(reps[-1], cl)]}
            lnv.close()
            if name == "fp64":
                ctx.release_cache()
        ctx.close()
        del S, H, L, L0, pS, pL
        torch.cuda.empty_cache()
        rows.append(row)
        print(json.dumps({"sub_batch": q, **{k: v for k, v in row.items()
                                             if k in ("cells", "atoms", "orbitals")},
                          "split_s_per_step": row["split"]["s_per_step"]}), flush=True)
    s_all = sum(r["split"]["s_per_step"] for r in rows)
    f_all = sum(r["split"]["gflops"] * r["split"]["s_per_step"] for r in rows)
    first = rows[0]
    print(json.dumps({
        "mode": "batch_c4",
        "workload": "32 cells of 500-8000 atoms (seeds 3-34), densities 0.03-0.06 atoms/A^3, "
                    "r_L 12-16 bohr, species 5/9/13 mixed per atom",
        "cells": len(cells), "atoms": int(sum(c[0].n_atoms for c in cells)),
        "sub_batches": len(rows), "sub_batch_atoms_max": args.c4_atoms,
        "split": {"s_per_step_all_cells": s_all, "gflops": f_all / s_all,
                  "dtype": "bf16x3 split, fp32 accumulate, fp64 traces", "graphs": True},
        "first_sub_batch": {"atoms": first["atoms"], "split_s_per_step": first["split"]["s_per_step"],
                            "fp64_s_per_step": first["fp64"]["s_per_step"],
                            "speedup": first["fp64"]["s_per_step"] / first["split"]["s_per_step"],
                            "energy_diff_per_atom_max": max(
                                abs(a - b) for a, b in zip(first["split"]["energy_per_atom"],
                                                           first["fp64"]["energy_per_atom"]))},
        "rows": rows, "input_wait_seconds": t_gen, "seconds": time.perf_counter() - t0}),
        flush=True)
    pool.shutdown()


def make_inputs(ncell):
    from paper_2205_08941_gb300 import inputs as I
    cell = I.diamond_cell(ncell, a=WORKLOAD["a_bohr"], sigma=WORKLOAD["sigma_bohr"],
                          seed=WORKLOAD["seed"], norb=9)
    S, H = I.overlap_hamiltonian(cell, I.silicon_model(WORKLOAD["r_S"]))
    return cell, S, H


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------- oracle sample

def oracle_sample(cell, Spb, Hpb, stride=64, reps=1):
    """The CPU oracle, as it stands, on a bounded sample of the same workload: the products
    of one LNV trial evaluation (X = LS, Y = LH in full; U = SX, R1 = UY, R3 = UX on every
    `stride`-th atom row).  Returns (GFLOP/s, seconds, flops, threads, description)."""
    import oracle as O
    from paper_2205_08941_gb300 import inputs as I
    rS, rL = WORKLOAD["r_S"], WORKLOAD["r_L"]
    pS, pL = O.Pattern.of_cell(cell, rS), O.Pattern.of_cell(cell, rL)
    pX, pU = O.Pattern.of_cell(cell, rL + rS), O.Pattern.of_cell(cell, 2 * rS + rL)
    S, H = O.scatter(pS, Spb), O.scatter(pS, Hpb)
    L = O.scatter(pL, I.random_blocks(cell, rL, 77)) * 0.01
    rows = np.arange(0, cell.n_atoms, stride, dtype=np.int32)
    flops = (O.triplets(pL, pS, pX)[1] * 2 + O.triplets(pS, pX, pU, rows)[1]
             + 2 * O.triplets(pU, pX, pL, rows)[1])
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        X = O.bsmm(1.0, pL, L, pS, S, 0.0, pX)
        Y = O.bsmm(1.0, pL, L, pS, H, 0.0, pX)
        U = O.bsmm(1.0, pS, S, pX, X, 0.0, pU, rows=rows)
        O.bsmm(1.0, pU, U, pX, Y, 0.0, pL, rows=rows)
        O.bsmm(1.0, pU, U, pX, X, 0.0, pL, rows=rows)
        times.append(time.perf_counter() - t0)
    desc = (f"oracle products of one LNV trial evaluation: X=LS, Y=LH full, U=SX, R1=UY, "
            f"R3=UX on {rows.shape[0]} of {cell.n_atoms} output atom rows "
            f"({flops / 1e9:.1f} GFLOP)")
    return flops / min(times) / 1e9, times, flops, O.num_threads(), desc


def oracle_sample_rows(cell, Spb, Hpb, stride):
    """The oracle's five trial-evaluation products restricted to every `stride`-th output
    atom row (all five, X and Y included): the same code and per-triplet work as
    oracle_sample, in a sample small enough for one core.  Rows of X outside the sample
    stay zero, which changes no operation count.  Returns (GFLOP/s, seconds, threads,
    description)."""
    import oracle as O
    from paper_2205_08941_gb300 import inputs as I
    rS, rL = WORKLOAD["r_S"], WORKLOAD["r_L"]
    pS, pL = O.Pattern.of_cell(cell, rS), O.Pattern.of_cell(cell, rL)
    pX, pU = O.Pattern.of_cell(cell, rL + rS), O.Pattern.of_cell(cell, 2 * rS + rL)
    S, H = O.scatter(pS, Spb), O.scatter(pS, Hpb)
    L = O.scatter(pL, I.random_blocks(cell, rL, 77)) * 0.01
    rows = np.arange(0, cell.n_atoms, stride, dtype=np.int32)
    flops = (O.triplets(pL, pS, pX, rows)[1] * 2 + O.triplets(pS, pX, pU, rows)[1]
             + 2 * O.triplets(pU, pX, pL, rows)[1])
    t0 = time.perf_counter()
    X = O.bsmm(1.0, pL, L, pS, S, 0.0, pX, rows=rows)
    Y = O.bsmm(1.0, pL, L, pS, H, 0.0, pX, rows=rows)
    U = O.bsmm(1.0, pS, S, pX, X, 0.0, pU, rows=rows)
    O.bsmm(1.0, pU, U, pX, Y, 0.0, pL, rows=rows)
    O.bsmm(1.0, pU, U, pX, X, 0.0, pL, rows=rows)
    sec = time.perf_counter() - t0
    desc = (f"oracle products of one LNV trial evaluation (X=LS, Y=LH, U=SX, R1=UY, R3=UX) "
            f"on {rows.shape[0]} of {cell.n_atoms} output atom rows ({flops / 1e9:.1f} GFLOP)")
    return flops / sec / 1e9, sec, O.num_threads(), desc


def cpu_one_core(ncell, stride=128):
    """cpu_baseline on one host core: the oracle in a child process with OMP_NUM_THREADS=1
    (its OpenMP pool is sized at start-up).  Returns a dict, or None if the child failed."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "c, s, h = bench.make_inputs(%d); "
            "g, sec, th, d = bench.oracle_sample_rows(c, s, h, %d); "
            "print(json.dumps([g, sec, th, d]))") % (ROOT, ncell, stride)
    env = dict(os.environ, OMP_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True,
                           text=True, timeout=600)
        g, sec, th, d = json.loads(r.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError):
        return None
    return {"value": g, "unit": "GFLOP/s", "cores": th, "kind": "oracle", "sample": d,
            "seconds": sec}


def split_oracle_check(dev, steps=3):
    """Split-BF16 LNV against the FP64 oracle on the 512-atom SZP cell (the benchmark's
    recipe at 1/8 of the atoms, where the oracle runs LNV steps in seconds): both start from
    the oracle's Palser-Manolopoulos L after eight Hotelling steps; after each step the
    energy difference per atom and ||L - L_oracle|| / ||L_oracle||.  Returns a dict."""
    import torch

    import oracle as O
    from paper_2205_08941_gb300 import cq
    from paper_2205_08941_gb300 import inputs as I
    rS, rL = WORKLOAD["r_S"], WORKLOAD["r_L"]
    cell = I.diamond_cell(4, a=WORKLOAD["a_bohr"], sigma=WORKLOAD["sigma_bohr"],
                          seed=WORKLOAD["seed"], norb=9)
    Spb, Hpb = I.overlap_hamiltonian(cell, I.silicon_model(rS))
    oS, oL = O.Pattern.of_cell(cell, rS), O.Pattern.of_cell(cell, rL)
    oX, oU = O.Pattern.of_cell(cell, rL + rS), O.Pattern.of_cell(cell, 2 * rS + rL)
    S_o, H_o = O.scatter(oS, Spb), O.scatter(oS, Hpb)
    T_o = O.hotelling_init(oS, S_o, oL)
    for _ in range(8):
        T_o, _ = O.hotelling_step(oS, S_o, oL, T_o, oX)
    n_e = 4.0 * cell.n_atoms
    L0 = O.pm_guess(oS, S_o, H_o, oL, T_o, oX, oL, n_e / 2)
    lo = O.LNV(oS, S_o, H_o, oL, L0, n_e, oX, oU)
    ctx = cq.Context(dev)
    t = lambda a, dt: torch.tensor(a, dtype=dt, device=f"cuda:{dev}")
    pos, nb = t(cell.pos, torch.float64), t(cell.nb, torch.int32)
    pS, pL = ctx.pattern(pos, cell.box, nb, rS), ctx.pattern(pos, cell.box, nb, rL)
    up = lambda p, pb: ctx.scatter(p, t(pb.i, torch.int32), t(pb.j, torch.int32),
                                   t(pb.off, torch.int64), t(pb.values, torch.float64))
    S, H = up(pS, Spb), up(pS, Hpb)
    # the same start on the GPU: oracle values placed block by block (same pattern order)
    _, col, off, _ = pL.export()
    sizes = np.diff(oL.off)
    idx = np.repeat(off.cpu().numpy() - oL.off[:-1], sizes) + np.arange(int(oL.off[-1]))
    idx = t(idx, torch.int64)
    L = ctx.zeros(pL)
    L[idx] = t(L0, torch.float64)
    lg = ctx.lnv(pS, S, H, pL, L, n_e, prec=cq.CQ_SPLIT_BF16X3)
    rows = []
    for _ in range(steps):
        ro, rg = lo.step(), lg.step()
        Lg = L[idx].cpu().numpy()
        rows.append({"energy_err_per_atom": abs(rg["energy"] - ro["E"]) / cell.n_atoms,
                     "L_rel_err": float(np.linalg.norm(Lg - lo.L) / np.linalg.norm(lo.L))})
    lg.close()
    ctx.close()
    return {"workload": workload_name(cell.n_atoms), "steps": steps, "per_step": rows,
            "energy_err_per_atom": rows[-1]["energy_err_per_atom"],
            "L_rel_err": rows[-1]["L_rel_err"]}


def bench_config(cell, args, world):
    """The workload of the bench line, the same for both arms."""
    return dict(WORKLOAD, workload=workload_name(cell.n_atoms), ncell=args.ncell,
                n_atoms=cell.n_atoms, n_electrons=4 * cell.n_atoms,
                parallelism=f"replicas x{world}",
                l2="inputs larger than L2 (U, Z 6.9 GB each)")


def run_reference(args, rank, world):
    if rank != 0:
        return
    cell, Spb, Hpb = make_inputs(args.ncell)
    sample = None
    vals, secs = [], []
    for k in range(args.warmup + args.steps):
        g, t, f, cores, desc = oracle_sample(cell, Spb, Hpb)
        if k >= args.warmup:
            vals.append(g)
            secs.append(t[0])
        sample = (cores, desc)
    v = sum(vals) / len(vals)
    line = {"impl": "reference", "metric": METRIC,
            "value": v, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": bench_config(cell, args, world),
            "cpu_baseline": {"value": v, "unit": "GFLOP/s", "cores": sample[0],
                             "kind": "oracle", "sample": sample[1]},
            "e2e": {"value": v, "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------- CUDA path

def run_cq(args, rank, world, local_rank):
    import torch

    from paper_2205_08941_gb300 import build as B
    B.build()
    from paper_2205_08941_gb300 import cq

    dev = local_rank
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    rep = Replicas(dist, torch.device("cuda", dev))
    barrier = rep.barrier

    cell, Spb, Hpb = make_inputs(args.ncell)
    ctx = cq.Context(dev)
    t = lambda a, dt: torch.tensor(a, dtype=dt, device=f"cuda:{dev}")
    pos, nb = t(cell.pos, torch.float64), t(cell.nb, torch.int32)
    rS, rL = WORKLOAD["r_S"], WORKLOAD["r_L"]
    pS = ctx.pattern(pos, cell.box, nb, rS)
    pL = ctx.pattern(pos, cell.box, nb, rL)

    def up(p, pb):
        return ctx.scatter(p, t(pb.i, torch.int32), t(pb.j, torch.int32),
                           t(pb.off, torch.int64), t(pb.values, torch.float64))

    S, H = up(pS, Spb), up(pS, Hpb)
    T = ctx.zeros(pL)
    ctx.hotelling_init(pS, S, pL, T)
    resid = [ctx.hotelling_step(pS, S, pL, T) for _ in range(args.hotelling_steps)]
    n_e = 4.0 * cell.n_atoms
    L = ctx.zeros(pL)
    ctx.pm_guess(pS, S, H, pL, T, pL, L, n_e / 2.0)
    del T
    first_prec = cq.CQ_SPLIT_BF16X3 if args.only_split else cq.CQ_FP64
    lnv = ctx.lnv(pS, S, H, pL, L, n_e, prec=first_prec)
    stream = torch.cuda.current_stream(dev)

    def timed(nsteps, label):
        """K timed steps on the device: CUDA events on the context's stream, clocks sampled,
        product-kernel launches timed by the library."""
        ctx.set_timing(True)
        ctx.kernel_stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clocks = ClockSampler(dev)
        barrier()
        launches0 = cq.kernel_launches()
        clocks.start()
        e0.record(stream)
        reps = [lnv.step() for _ in range(nsteps)]
        e1.record(stream)
        barrier()
        clk = clocks.stop()
        ms = rep.max(e0.elapsed_time(e1))
        flops_all = rep.sum(sum(x["flops"] for x in reps))
        stats = ctx.kernel_stats()
        ctx.set_timing(False)
        return {"reps": reps, "ms": ms, "clk": clk, "stats": stats, "flops_all": flops_all,
                "launches": cq.kernel_launches() - launches0}

    for _ in range(args.warmup):
        lnv.step()
    L0 = L.clone()
    res = {}
    peak_fp64 = ctx.peak_fp64()
    if not args.only_split:
        lnv.set_precision(cq.CQ_FP64)  # fresh search direction at L0
        res["fp64"] = timed(args.steps, "fp64")
        E_fp64, L_fp64 = res["fp64"]["reps"][-1]["energy"], L.clone()

    e2e = None
    if not args.no_e2e and not args.only_split:
        # end to end through the public API over the same K steps from the same start L0:
        # each step copies the iterate L in from pinned host memory, runs cq_lnv_step and
        # reads L and the step's scalars back
        L.copy_(L0)
        lnv.set_precision(cq.CQ_FP64)  # the same fresh start as the timed FP64 steps
        L_host = torch.empty(L.shape, dtype=torch.float64, pin_memory=True)
        L_host.copy_(L)
        torch.cuda.synchronize()
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e2.record(stream)
        fl2 = 0.0
        for _ in range(args.steps):
            L.copy_(L_host, non_blocking=True)
            r = lnv.step()
            L_host.copy_(L, non_blocking=True)
            fl2 += r["flops"]
        e3.record(stream)
        barrier()
        ms2 = rep.max(e2.elapsed_time(e3))
        e2e = {"value": rep.sum(fl2) / (ms2 * 1e-3) / 1e9, "unit": "GFLOP/s",
               "h2d_bytes_per_step": int(L.numel() * 8),
               "d2h_bytes_per_step": int(L.numel() * 8 + 96),
               "ms_per_step": ms2 / args.steps, "steps": args.steps,
               "same_steps_as_value": True}

    split = None
    if not args.no_split:
        L.copy_(L0)
        lnv.set_precision(cq.CQ_SPLIT_BF16X3)
        for _ in range(args.warmup):
            lnv.step()
        L.copy_(L0)
        lnv.set_precision(cq.CQ_SPLIT_BF16X3)
        res["split"] = timed(args.steps, "split")
        r = res["split"]
        n_launch, kern_ms, kern_flops, mma_flops = r["stats"]
        peaks = measured_peaks()
        bf16 = (peaks or {}).get("bf16_tflops")
        split = {"value": r["flops_all"] / (r["ms"] * 1e-3) / 1e9, "unit": "GFLOP/s",
                 "dtype": "bf16x3 split, fp32 accumulate, fp64 traces",
                 "ms_per_step": r["ms"] / args.steps, "s_per_lnv_step": r["ms"] / args.steps / 1e3,
                 "roofline": {"bound": "tensor", "kernel": "k_bsmm_split",
                              "achieved": mma_flops / (kern_ms * 1e-3) / 1e12 if kern_ms else None,
                              "peak": bf16 or BF16_FALLBACK_TFLOPS, "unit": "TFLOP/s",
                              "peak_source": "MEASURED_PEAKS.json bf16_tflops" if bf16 else
                              "profiling-recipe fallback (1.9 PFLOP/s bf16)",
                              "useful_tflops": kern_flops / (kern_ms * 1e-3) / 1e12 if kern_ms else None,
                              "launches": n_launch, "kernel_ms": kern_ms,
                              "kernel_share": kern_ms / r["ms"] if r["ms"] else None,
                              "traffic": SPLIT_TRAFFIC_PER_LAUNCH if cell.n_atoms == 4096 else None,
                              "traffic_source": TRAFFIC_SOURCE},
                 "clocks": r["clk"], "gpu_launches": int(r["launches"]),
                 "lnv": [{k: x[k] for k in ("energy", "n_elec", "gnorm", "n_corr")}
                         for x in r["reps"]]}
        split["roofline"]["frac"] = (split["roofline"]["achieved"] / split["roofline"]["peak"]
                                     if split["roofline"]["achieved"] else None)
        # useful work at the method's own cost: six BF16 products per FP64-equivalent flop
        uf = split["roofline"]["useful_tflops"]
        split["roofline"]["useful_frac"] = (6.0 * uf / split["roofline"]["peak"]) if uf else None
        if "fp64" in res:
            E_split = r["reps"][-1]["energy"]
            split["energy_err_per_atom_vs_fp64"] = abs(E_split - E_fp64) / cell.n_atoms
            split["L_rel_diff_vs_fp64"] = float(torch.linalg.vector_norm(L - L_fp64) /
                                                torch.linalg.vector_norm(L_fp64))
            split["speedup_vs_fp64_step"] = (res["fp64"]["ms"] / r["ms"])

    emu = None
    if not args.no_emu and not args.only_split:
        # FP64-accurate products on the tensor cores: the same K steps from the same L0
        L.copy_(L0)
        lnv.set_precision(cq.CQ_FP64_EMU)
        k_emu = min(args.steps, 3)  # an extra leg: at most three steps keep the bench short
        res["emu"] = timed(k_emu, "emu")
        r = res["emu"]
        n_launch, kern_ms, kern_flops, mma_flops = r["stats"]
        peaks = measured_peaks()
        bf16 = (peaks or {}).get("bf16_tflops")
        # FP64 time of the same work over the emulated time: the two legs' useful-flop rates
        # (the emulated leg times at most three steps from L0, the FP64 leg all K, and early
        # steps run more products than late ones, so their times per step do not compare)
        fp64_rate = (res["fp64"]["flops_all"] / res["fp64"]["ms"]
                     if "fp64" in res and res["fp64"]["ms"] > 0 else None)
        emu = {"value": r["flops_all"] / (r["ms"] * 1e-3) / 1e9, "unit": "GFLOP/s",
               "dtype": "f64 emulated: 8 bf16 digit planes, exact level sums", "steps": k_emu,
               "s_per_lnv_step": r["ms"] / k_emu / 1e3,
               "speedup_vs_fp64_step": ((r["flops_all"] / r["ms"]) / fp64_rate
                                        if fp64_rate and r["ms"] > 0 else None),
               "roofline": {"bound": "tensor", "kernel": "k_bsmm_emu",
                            "achieved": mma_flops / (kern_ms * 1e-3) / 1e12 if kern_ms else None,
                            "peak": bf16 or BF16_FALLBACK_TFLOPS, "unit": "TFLOP/s",
                            "useful_tflops": kern_flops / (kern_ms * 1e-3) / 1e12 if kern_ms else None,
                            "launches": n_launch, "kernel_ms": kern_ms,
                            "kernel_share": kern_ms / r["ms"] if r["ms"] else None,
                            "traffic": EMU_TRAFFIC_PER_LAUNCH if cell.n_atoms == 4096 else None,
                            "traffic_source": TRAFFIC_SOURCE},
               "clocks": r["clk"], "gpu_launches": int(r["launches"])}
        emu["roofline"]["frac"] = (emu["roofline"]["achieved"] / emu["roofline"]["peak"]
                                   if emu["roofline"]["achieved"] else None)
        if "fp64" in res:
            emu["energy_diff_per_atom_vs_fp64"] = abs(r["reps"][-1]["energy"] - E_fp64) / cell.n_atoms
            emu["L_rel_diff_vs_fp64"] = float(torch.linalg.vector_norm(L - L_fp64) /
                                              torch.linalg.vector_norm(L_fp64))
            emu["same_step_decisions_as_fp64"] = all(
                (a["restart"], a["fallback"], a["n_corr"]) == (b["restart"], b["fallback"], b["n_corr"])
                for a, b in zip(r["reps"], res["fp64"]["reps"]))
            # the FP64 trajectory after the same number of steps
            E_k = res["fp64"]["reps"][k_emu - 1]["energy"]
            emu["energy_diff_per_atom_vs_fp64"] = abs(r["reps"][-1]["energy"] - E_k) / cell.n_atoms
            emu.pop("L_rel_diff_vs_fp64", None)

    batched = None
    if not args.no_batch:
        batched = run_batch(args, dev, rep)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        g, times, f, cores, desc = oracle_sample(cell, Spb, Hpb)
        cpu = {"value": g, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
               "sample": desc, "seconds": min(times),
               "one_core": cpu_one_core(args.ncell)}

    if split is not None and rank == 0 and world == 1 and not args.no_oracle_check:
        split["oracle_check"] = split_oracle_check(dev)

    conv = None
    if rank == 0 and world == 1 and not args.no_converge and not args.only_split:
        conv = converge_quick(args, dev)

    if rank == 0:
        main = res.get("fp64") or res.get("split")
        n_launch, kern_ms, kern_flops, mma_flops = main["stats"]
        ms = main["ms"]
        achieved = kern_flops / (kern_ms * 1e-3) / 1e12 if kern_ms > 0 else None
        line = {
            "metric": METRIC,
            "value": main["flops_all"] / (ms * 1e-3) / 1e9, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "s_per_lnv_step": ms / args.steps / 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if "fp64" in res else "bf16x3", "data": "synthetic",
            "config": bench_config(cell, args, world),
            "hotelling_resid": resid[-1] if resid else None,
            "roofline": {"bound": "alu", "kernel": "k_bsmm_f64_uniform",
                         "achieved": achieved, "peak": peak_fp64 / 1e12, "unit": "TFLOP/s",
                         "frac": (achieved / (peak_fp64 / 1e12)) if achieved else None,
                         "traffic": FP64_TRAFFIC_PER_LAUNCH if cell.n_atoms == 4096 else None,
                         "traffic_source": TRAFFIC_SOURCE,
                         "peak_source": "in-library FP64 probe (best of FMA and DMMA chains)",
                         "launches": n_launch, "kernel_ms": kern_ms,
                         "kernel_share": kern_ms / ms if ms > 0 else None},
            "lnv": [{k: x[k] for k in ("energy", "n_elec", "gnorm", "alpha", "n_corr",
                                       "n_products")} for x in main["reps"]],
            "batched": batched,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": main["clk"],
            "gpu_launches": int(main["launches"]),
        }
        if "fp64" not in res:
            line["roofline"] = split["roofline"]
        if emu is not None:
            line["fp64_emu"] = emu
        if conv is not None:
            line["converge"] = conv
        if split is not None:
            # last, and compact, so that a reader of the line's tail sees the mixed leg
            split.pop("lnv", None)
            line["split"] = split
        print(json.dumps(line), flush=True)
    lnv.close()
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------- convergence criteria

def run_until(lnv, gtol, cap, trace=None, t0=0.0, fp64=True, stall=None, de_tol=None):
    """LNV steps until the RMS gradient is <= gtol (at most cap steps), or, with stall, until
    it has fallen by less than the factor stall over two steps -- split-BF16 gradients stop
    improving near their rounding floor (about 1e-6 RMS on the 4096-atom cell) -- or, with
    de_tol, until the energy changes by less than de_tol in one step.  trace gets (seconds
    since t0, energy, RMS gradient, whether the step's products were FP64) per step.
    Returns (steps, last report)."""
    it, st = 0, lnv.state()
    hist = [st["gnorm"]]
    while st["gnorm"] > gtol and it < cap:
        e_prev = st["energy"]
        st = lnv.step()
        it += 1
        hist.append(st["gnorm"])
        if trace is not None:
            trace.append((time.perf_counter() - t0, st["energy"], st["gnorm"], fp64))
        if stall is not None and len(hist) >= 3 and hist[-1] > stall * hist[-3]:
            break
        if de_tol is not None and abs(st["energy"] - e_prev) < de_tol:
            break
    return it, st


def settled(trace, e_ref, tol):
    """Seconds until every later FP64-product energy of the trace stays within tol of e_ref
    (split-product energies carry the split's bias and do not count); None if never."""
    fp = [x for x in trace if x[3]]
    for k in range(len(fp)):
        if all(abs(y[1] - e_ref) <= tol for y in fp[k:]):
            return fp[k][0]
    return None


def de_stop(trace, tol):
    """The intrinsic stop rule: the first FP64 step whose energy differs from the previous
    FP64 step's by less than tol, as (seconds, energy); (None, None) if none."""
    fp = [x for x in trace if x[3]]
    for k in range(1, len(fp)):
        if abs(fp[k][1] - fp[k - 1][1]) < tol:
            return fp[k][0], fp[k][1]
    return None, None


def cell_setup(ctx, dev):
    """setup(cell, S pair blocks, H pair blocks, hsteps) on ctx: patterns P_S, P_L, S and H
    on the device, and T ~ S^-1 from hsteps Hotelling steps."""
    import torch
    t = lambda a, dt: torch.tensor(a, dtype=dt, device=f"cuda:{dev}")
    rS, rL = WORKLOAD["r_S"], WORKLOAD["r_L"]

    def setup(cell, Spb, Hpb, hsteps=12):
        pos, nb = t(cell.pos, torch.float64), t(cell.nb, torch.int32)
        pS, pL = ctx.pattern(pos, cell.box, nb, rS), ctx.pattern(pos, cell.box, nb, rL)
        up = lambda p, pb: ctx.scatter(p, t(pb.i, torch.int32), t(pb.j, torch.int32),
                                       t(pb.off, torch.int64), t(pb.values, torch.float64))
        S, H = up(pS, Spb), up(pS, Hpb)
        T = ctx.zeros(pL)
        ctx.hotelling_init(pS, S, pL, T)
        for _ in range(hsteps):
            ctx.hotelling_step(pS, S, pL, T)
        return pS, pL, S, H, T
    return setup


def train_guess(ctx, setup, train_cells, train_ncell, train_split):
    """The learned start's network trained on converged L of small thermally displaced
    cells; returns (guess, description of the training)."""
    import torch

    from paper_2205_08941_gb300 import cq, learned
    from paper_2205_08941_gb300 import inputs as I
    rS = WORKLOAD["r_S"]
    # training set: converged L of small thermally displaced cells (seeds 1000 + k, jitter
    # sigma ~ U[0.1, 0.3] bohr), solved in FP64 to RMS 1e-7 or, with --train-split, by
    # split-BF16 steps to RMS 1e-6 (the targets only have to make a good start)
    t0 = time.perf_counter()
    rng = np.random.default_rng(1000)
    samples, keep = [], []
    train_prec = cq.CQ_SPLIT_BF16X3 if train_split else cq.CQ_FP64
    for k in range(train_cells):
        c = I.diamond_cell(train_ncell, a=WORKLOAD["a_bohr"],
                           sigma=float(rng.uniform(0.1, 0.3)), seed=1000 + k, norb=9)
        s_, h_ = I.overlap_hamiltonian(c, I.silicon_model(rS))
        pS, pL, S, H, T = setup(c, s_, h_)
        L = ctx.zeros(pL)
        ctx.pm_guess(pS, S, H, pL, T, pL, L, 2.0 * c.n_atoms)
        lnv = ctx.lnv(pS, S, H, pL, L, 4.0 * c.n_atoms, prec=train_prec)
        if train_split:
            run_until(lnv, 1e-6, 80, stall=0.9)
        else:
            run_until(lnv, 1e-7, 80)
        lnv.close()
        samples.append((pL, L))
        del pS, S, H, T
        if (k + 1) % 16 == 0:
            ctx.release_cache()  # every cell has its own patterns: drop their plans
    t_data = time.perf_counter() - t0
    guess = cq.Guess(ctx, seed=11)
    desc, targ = learned.training_set(guess, samples)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    epochs = 60
    hist = learned.train(guess, desc, targ, epochs=epochs, batch=4096, lr=2e-3, lr_decay=0.96)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t1
    t_train = time.perf_counter() - t0
    n_samples = int(desc.shape[0])
    # MLP work of the fit: forward 2 sum(d_l d_l+1) flops per sample, backward twice that
    dims = (64, 256, 256, 256, 81)
    fwd = 2.0 * sum(a * b for a, b in zip(dims, dims[1:]))
    mlp_tflops = 3.0 * fwd * n_samples * epochs / t_fit / 1e12
    peaks = measured_peaks()
    bf16 = (peaks or {}).get("bf16_tflops")
    training = {"cells": train_cells, "atoms_per_cell": 8 * train_ncell ** 3,
                "solver": "split-BF16 to RMS 1e-6" if train_split else "FP64 to RMS 1e-7",
                "samples": n_samples, "epochs": epochs, "seconds": t_train,
                "data_seconds": t_data, "fit_seconds": t_fit,
                "loss_first_last": [hist[0], hist[-1]],
                "mlp_tflops": mlp_tflops,
                "mlp_frac_of_bf16_peak": mlp_tflops / bf16 if bf16 else None}
    del samples, keep, desc, targ
    return guess, training


def converge_quick(args, dev):
    """The target criterion on the 4096-atom cell in the default bench: seconds until the
    energy stays within 1e-6 Ha/atom of the FP64 solution,
    (a) plain: PM start, FP64 LNV until the energy changes by less than 1e-7 Ha/atom in one
        step -- its final energy is the reference (6e-8 Ha/atom from the RMS-1e-8 solution);
    (b) learned start (network trained on six 216-atom cells), split-BF16 LNV to its
        rounding floor, then FP64 steps to the same stop rule.
    Times exclude patterns, the Hotelling inverse and the one-off training."""
    import torch

    from paper_2205_08941_gb300 import cq, learned
    ctx = cq.Context(dev)
    setup = cell_setup(ctx, dev)
    guess, training = train_guess(ctx, setup, 6, 3, False)
    ctx.release_cache()
    cell, Spb, Hpb = make_inputs(args.ncell)
    n_at = cell.n_atoms
    n_e = 4.0 * n_at
    pS, pL, S, H, T = setup(cell, Spb, Hpb, args.hotelling_steps)
    de = 1e-7 * n_at
    L = ctx.zeros(pL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.pm_guess(pS, S, H, pL, T, pL, L, n_e / 2.0)
    lnv = ctx.lnv(pS, S, H, pL, L, n_e)
    tr_a = []
    it_a, st_a = run_until(lnv, 1e-8, 120, tr_a, t0, de_tol=de)
    torch.cuda.synchronize()
    t_a = time.perf_counter() - t0
    lnv.close()
    L2 = ctx.zeros(pL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lnv, used, info = learned.guarded_start(ctx, guess, pS, S, H, pL, T, pL, L2, n_e,
                                            prec=cq.CQ_SPLIT_BF16X3)
    tr_b = []
    it_b1, st_b1 = run_until(lnv, 1e-6, 120, tr_b, t0, fp64=False, stall=0.9)
    lnv.set_precision(cq.CQ_FP64)
    it_b2, st_b2 = run_until(lnv, 1e-8, 60, tr_b, t0, de_tol=de)
    torch.cuda.synchronize()
    t_b = time.perf_counter() - t0
    lnv.close()
    e_ref = st_a["energy"]
    ta6, tb6 = settled(tr_a, e_ref, 1e-6 * n_at), settled(tr_b, e_ref, 1e-6 * n_at)
    out = {"criterion": "energy within 1e-6 Ha/atom of the FP64 solution (plain FP64 LNV "
                        "stopped when its energy changes by < 1e-7 Ha/atom per step)",
           "plain_fp64_seconds": ta6, "learned_split_seconds": tb6,
           "speedup": (ta6 / tb6) if ta6 and tb6 else None,
           "plain_fp64": {"seconds_to_stop": t_a, "steps": it_a, "gnorm": st_a["gnorm"]},
           "learned_split_then_fp64": {"seconds_to_stop": t_b, "split_steps": it_b1,
                                       "fp64_steps": it_b2, "gnorm": st_b2["gnorm"],
                                       "energy_diff_per_atom":
                                           abs(st_b2["energy"] - e_ref) / n_at,
                                       "learned_start_used": used,
                                       "gnorm_start": info["gnorm_learned"],
                                       "gnorm_pm_start": info["gnorm_pm"]},
           "training": {k: training[k] for k in ("cells", "atoms_per_cell", "samples",
                                                 "seconds", "fit_seconds", "mlp_tflops",
                                                 "mlp_frac_of_bf16_peak", "loss_first_last")}}
    guess.close()
    ctx.close()
    return out


def run_converge(args, dev):
    """Full minimisations on the 4096-atom cell, both to RMS gradient 1e-8:
    (a) plain: PM start, FP64 LNV;
    (b) learned: network trained on converged 216-atom cells (thermal jitter 0.1-0.3 bohr),
        guarded learned start, split-BF16 LNV to RMS gradient 1e-6 (or until it stops
        improving: less than 10% over two steps), FP64 refinement.
    Reported for three criteria: RMS gradient 1e-8; energy settled within 1e-6 Ha/atom of
    the converged FP64 energy (FP64-product energies only); the intrinsic rule "FP64 energy
    change per step below 1e-7 Ha/atom".  Times exclude pattern/task-list construction
    (shared, cached) and the one-off training."""
    import torch

    from paper_2205_08941_gb300 import build as B
    B.build()
    from paper_2205_08941_gb300 import cq, learned
    from paper_2205_08941_gb300 import inputs as I
    torch.cuda.set_device(dev)
    ctx = cq.Context(dev)
    setup = cell_setup(ctx, dev)

    def rel(x, ref):
        return float(torch.linalg.vector_norm(x - ref) / torch.linalg.vector_norm(ref))

    def run(lnv, gtol, cap, trace=None, t0=0.0, fp64=True, stall=None):
        return run_until(lnv, gtol, cap, trace, t0, fp64, stall)

    guess, training = train_guess(ctx, setup, args.train_cells, args.train_ncell,
                                  args.train_split)
    cell, Spb, Hpb = make_inputs(args.ncell)
    n_e = 4.0 * cell.n_atoms
    pS, pL, S, H, T = setup(cell, Spb, Hpb, args.hotelling_steps)
    if args.apply_only:
        # the network trained on 216-atom cells applied to this cell, then split-BF16 steps
        L2 = ctx.zeros(pL)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lnv, used, info = learned.guarded_start(ctx, guess, pS, S, H, pL, T, pL, L2, n_e,
                                                prec=cq.CQ_SPLIT_BF16X3)
        torch.cuda.synchronize()
        t_start = time.perf_counter() - t0
        tr = []
        it, st = run(lnv, 1e-6, 120, tr, t0, fp64=False, stall=0.9)
        torch.cuda.synchronize()
        t_all = time.perf_counter() - t0
        lnv.close()
        print(json.dumps({
            "mode": "learned_apply", "workload": workload_name(cell.n_atoms),
            "n_atoms": cell.n_atoms, "learned_start_used": used, "start": info,
            "start_seconds": t_start, "split_steps": it, "split_seconds": t_all - t_start,
            "gnorm": st["gnorm"], "energy_per_atom": st["energy"] / cell.n_atoms,
            "gnorm_trace": [x[2] for x in tr],
            "training": training}), flush=True)
        guess.close()
        ctx.close()
        return
    # (a) plain FP64 from the PM start
    L = ctx.zeros(pL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.pm_guess(pS, S, H, pL, T, pL, L, n_e / 2.0)
    lnv = ctx.lnv(pS, S, H, pL, L, n_e)
    tr_a = []
    it_a, st_a = run(lnv, 1e-8, 120, tr_a, t0)
    torch.cuda.synchronize()
    t_a = time.perf_counter() - t0
    lnv.close()
    # (b) learned start, split-BF16 steps, FP64 refinement
    L2 = ctx.zeros(pL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lnv, used, info = learned.guarded_start(ctx, guess, pS, S, H, pL, T, pL, L2, n_e,
                                            prec=cq.CQ_SPLIT_BF16X3)
    tr_b = []
    it_b1, st_b1 = run(lnv, 1e-6, 120, tr_b, t0, fp64=False, stall=0.9)
    t_b1 = time.perf_counter() - t0
    L2_split = L2.clone()  # the split-only solution, compared after the timings
    lnv.set_precision(cq.CQ_FP64)
    it_b2, st_b2 = run(lnv, 1e-8, 60, tr_b, t0)
    torch.cuda.synchronize()
    t_b = time.perf_counter() - t0
    lnv.close()
    n_at = cell.n_atoms
    e_ref = st_a["energy"]
    ta6, tb6 = settled(tr_a, e_ref, 1e-6 * n_at), settled(tr_b, e_ref, 1e-6 * n_at)
    within = {"plain_seconds": ta6, "learned_split_seconds": tb6,
              "speedup": (ta6 / tb6) if ta6 and tb6 else None}
    (sa, ea), (sb, eb) = de_stop(tr_a, 1e-7 * n_at), de_stop(tr_b, 1e-7 * n_at)
    stop_rule = {"plain_seconds": sa, "plain_err_per_atom": abs(ea - e_ref) / n_at if ea else None,
                 "learned_split_seconds": sb,
                 "learned_split_err_per_atom": abs(eb - e_ref) / n_at if eb else None,
                 "speedup": (sa / sb) if sa and sb else None}
    line = {"mode": "converge", "workload": workload_name(cell.n_atoms), "n_atoms": cell.n_atoms,
            "gradient_target_rms": 1e-8,
            "plain_fp64": {"seconds": t_a, "steps": it_a, "energy": st_a["energy"],
                           "gnorm": st_a["gnorm"]},
            "learned_split_then_fp64": {
                "seconds": t_b, "split_steps": it_b1, "split_seconds": t_b1,
                "fp64_steps": it_b2, "energy": st_b2["energy"], "gnorm": st_b2["gnorm"],
                "learned_start_used": used, "start": info},
            "energy_diff_per_atom": abs(st_b2["energy"] - st_a["energy"]) / cell.n_atoms,
            "L_rel_diff": rel(L2, L),
            "split_only_vs_fp64": {  # split-BF16 solution at RMS gradient 1e-6, before refinement
                "energy_err_per_atom": abs(st_b1["energy"] - st_a["energy"]) / cell.n_atoms,
                "L_rel_diff": rel(L2_split, L)},
            "speedup": t_a / t_b,
            # the target criterion: energy within 1e-6 Ha/atom of the converged FP64 energy
            # (plain run at RMS gradient 1e-8), judged on FP64-product energies only
            "within_1e-6_per_atom": within,
            # intrinsic stopping rule for both: FP64 energy change per step < 1e-7 Ha/atom
            "stop_dE_1e-7_per_atom": stop_rule,
            "training": training}
    print(json.dumps(line), flush=True)
    guess.close()
    ctx.close()


def run_converge_emu(args, dev):
    """N1 end to end: the 4096-atom cell minimised to RMS gradient 1e-8 from the same PM start
    (a) with FP64 products and (b) with emulated-FP64 products on the tensor cores only (no
    FP64-pipe product anywhere in the solve).  Reports steps, seconds, the energies and
    their difference, and the relative difference of the two density matrices."""
    import torch

    from paper_2205_08941_gb300 import build as B
    B.build()
    from paper_2205_08941_gb300 import cq
    torch.cuda.set_device(dev)
    ctx = cq.Context(dev)
    setup = cell_setup(ctx, dev)
    cell, Spb, Hpb = make_inputs(args.ncell)
    n_at, n_e = cell.n_atoms, 4.0 * cell.n_atoms
    pS, pL, S, H, T = setup(cell, Spb, Hpb, args.hotelling_steps)
    L0 = ctx.zeros(pL)
    ctx.pm_guess(pS, S, H, pL, T, pL, L0, n_e / 2.0)
    del T
    out = {"mode": "converge_emu", "workload": workload_name(n_at), "gradient_target_rms": 1e-8}
    Ls = {}
    for name, prec in (("fp64", cq.CQ_FP64), ("emu", cq.CQ_FP64_EMU)):
        if prec != cq.CQ_FP64:
            ctx.release_cache()  # the FP64 task lists: the emulated steps need none
        L = L0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lnv = ctx.lnv(pS, S, H, pL, L, n_e, prec=prec)
        tr = []
        it, st = run_until(lnv, 1e-8, 80, tr, t0, fp64=True)
        torch.cuda.synchronize()
        out[name] = {"seconds": time.perf_counter() - t0, "steps": it, "energy": st["energy"],
                     "gnorm": st["gnorm"], "n_elec": st["n_elec"],
                     "gnorm_trace": [x[2] for x in tr]}
        lnv.close()
        Ls[name] = L
    out["energy_diff_per_atom"] = abs(out["emu"]["energy"] - out["fp64"]["energy"]) / n_at
    out["L_rel_diff"] = float(torch.linalg.vector_norm(Ls["emu"] - Ls["fp64"]) /
                              torch.linalg.vector_norm(Ls["fp64"]))
    out["speedup"] = out["fp64"]["seconds"] / out["emu"]["seconds"]
    print(json.dumps(out), flush=True)
    ctx.close()


def run_solvers(args, dev):
    """N4 and N2 at the benchmark's size.  Overlap inverse on P_L: 12 Hotelling steps against
    the least-squares inverse by CG (from the same T_0, up to 40 steps), residual ||I - ST||_F
    and seconds.  LNV from the same PM start (Hotelling T): plain against T-preconditioned
    directions, FP64 products, to RMS gradient 1e-8; steps, seconds, energies."""
    import torch

    from paper_2205_08941_gb300 import build as B
    B.build()
    from paper_2205_08941_gb300 import cq
    torch.cuda.set_device(dev)
    cell, Spb, Hpb = make_inputs(args.ncell)
    ctx = cq.Context(dev)
    t = lambda a, dt: torch.tensor(a, dtype=dt, device=f"cuda:{dev}")
    pos, nb = t(cell.pos, torch.float64), t(cell.nb, torch.int32)
    pS = ctx.pattern(pos, cell.box, nb, WORKLOAD["r_S"])
    pL = ctx.pattern(pos, cell.box, nb, WORKLOAD["r_L"])
    up = lambda p, pb: ctx.scatter(p, t(pb.i, torch.int32), t(pb.j, torch.int32),
                                   t(pb.off, torch.int64), t(pb.values, torch.float64))
    S, H = up(pS, Spb), up(pS, Hpb)
    n_e = 4.0 * cell.n_atoms
    out = {"mode": "solvers", "workload": workload_name(cell.n_atoms)}
    # overlap inverse: Hotelling against least-squares CG
    T = ctx.zeros(pL)
    ctx.hotelling_init(pS, S, pL, T)
    ctx.hotelling_step(pS, S, pL, T)  # task lists and scratch before the clock
    ctx.hotelling_init(pS, S, pL, T)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hres = [ctx.hotelling_step(pS, S, pL, T) for _ in range(12)]
    torch.cuda.synchronize()
    t_h = time.perf_counter() - t0
    Tc = ctx.zeros(pL)
    ctx.hotelling_init(pS, S, pL, Tc)
    ctx.overlap_inverse_cg(pS, S, pL, Tc, 1)
    ctx.hotelling_init(pS, S, pL, Tc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cres, cg = ctx.overlap_inverse_cg(pS, S, pL, Tc, 40, 1e-6)
    torch.cuda.synchronize()
    t_c = time.perf_counter() - t0
    # the Hotelling residual of the final T (one more step reports it)
    Th = T.clone()
    h_final = ctx.hotelling_step(pS, S, pL, Th)
    Tc2 = Tc.clone()
    c_final = ctx.hotelling_step(pS, S, pL, Tc2)
    del Th, Tc2
    out["overlap_inverse"] = {
        "hotelling": {"steps": 12, "seconds": t_h, "resid_final": h_final,
                      "resid_history": hres},
        "least_squares_cg": {"steps": len(cres) - 1, "seconds": t_c, "resid_final": c_final,
                             "resid_history": cres}}
    # LNV: plain against preconditioned, from the same PM start
    rows = {}
    for name in ("plain", "preconditioned"):
        L = ctx.zeros(pL)
        torch.cuda.synchronize()
        ctx.pm_guess(pS, S, H, pL, T, pL, L, n_e / 2.0)
        lnv = ctx.lnv(pS, S, H, pL, L, n_e)
        if name == "preconditioned":
            lnv.set_preconditioner(pL, T)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, st = run_until(lnv, 1e-8, 80)
        torch.cuda.synchronize()
        rows[name] = {"steps": it, "seconds": time.perf_counter() - t0, "gnorm": st["gnorm"],
                      "energy_per_atom": st["energy"] / cell.n_atoms,
                      "flops_per_step": lnv.step_flops()}
        lnv.close()
        del L
    rows["energy_diff_per_atom"] = abs(rows["plain"]["energy_per_atom"] -
                                       rows["preconditioned"]["energy_per_atom"])
    out["lnv_to_rms_1e-8"] = rows
    print(json.dumps(out), flush=True)
    ctx.close()


def run_sweep(args, dev):
    """Seconds per LNV step against the number of atoms, one GPU: for each cell size the
    patterns, Hotelling inverse and PM start are built (untimed), the LNV object takes two
    untimed steps, then one step is timed with CUDA events.  Split-BF16 at every size; FP64
    up to --sweep-fp64-max cells per edge (its step is ~7x longer)."""
    import torch

    from paper_2205_08941_gb300 import build as B
    B.build()
    from paper_2205_08941_gb300 import cq
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    t = lambda a, dt: torch.tensor(a, dtype=dt, device=f"cuda:{dev}")
    rows = []
    for ncell in [int(x) for x in args.sweep.split(",")]:
        cell, Spb, Hpb = make_inputs(ncell)
        n_e = 4.0 * cell.n_atoms
        precs = [("split", cq.CQ_SPLIT_BF16X3)]
        if ncell <= args.sweep_fp64_max:
            precs.append(("fp64", cq.CQ_FP64))
        row = {"ncell": ncell, "n_atoms": cell.n_atoms}
        for name, prec in precs:
            ctx = cq.Context(dev)
            pos, nb = t(cell.pos, torch.float64), t(cell.nb, torch.int32)
            pS = ctx.pattern(pos, cell.box, nb, WORKLOAD["r_S"])
            pL = ctx.pattern(pos, cell.box, nb, WORKLOAD["r_L"])
            up = lambda p, pb: ctx.scatter(p, t(pb.i, torch.int32), t(pb.j, torch.int32),
                                           t(pb.off, torch.int64), t(pb.values, torch.float64))
            S, H = up(pS, Spb), up(pS, Hpb)
            T = ctx.zeros(pL)
            ctx.hotelling_init(pS, S, pL, T)
            for _ in range(args.hotelling_steps):
                ctx.hotelling_step(pS, S, pL, T)
            L = ctx.zeros(pL)
            ctx.pm_guess(pS, S, H, pL, T, pL, L, n_e / 2.0)
            del T
            if prec != cq.CQ_FP64:
                ctx.release_cache()  # the set-up's FP64 task lists: tensor-core steps need none
            lnv = ctx.lnv(pS, S, H, pL, L, n_e, prec=prec)
            for _ in range(2):
                lnv.step()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            rep = lnv.step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            row[name] = {"s_per_step": ms / 1e3, "gflops": rep["flops"] / (ms * 1e-3) / 1e9,
                         "tflop_per_step": rep["flops"] / 1e12, "n_products": rep["n_products"],
                         "energy_per_atom": rep["energy"] / cell.n_atoms,
                         "gnorm": rep["gnorm"]}
            lnv.close()
            ctx.close()
            del S, H, L
            torch.cuda.empty_cache()
        rows.append(row)
        print(json.dumps(row), flush=True)
    base = rows[0]
    for r in rows:
        r["split_s_per_step_per_atom_rel"] = ((r["split"]["s_per_step"] / r["n_atoms"]) /
                                              (base["split"]["s_per_step"] / base["n_atoms"]))
    print(json.dumps({"mode": "sweep", "workload": "Si diamond SZP, a = 10.26 bohr, sigma 0.1, "
                      "r_S 14, r_L 16", "rows": rows}), flush=True)


PRODUCTS = {"X": ("r_L", "r_S", "r_X"), "U": ("r_S", "r_X", "r_U"), "R": ("r_U", "r_X", "r_L")}


def run_products(args, dev):
    """Kernel time of single block products of the LNV step's three kinds on the Si SZP cell,
    operands seeded N(0,1) blocks decaying with distance (inputs.random_blocks); only the
    matrices of the named products are made.  One untimed product per kind (it builds the
    plan), then --steps timed ones, timed by the library around its product kernels."""
    import torch

    from paper_2205_08941_gb300 import build as B
    B.build()
    from paper_2205_08941_gb300 import cq
    from paper_2205_08941_gb300 import inputs as I
    torch.cuda.set_device(dev)
    prec = {"fp64": cq.CQ_FP64, "split": cq.CQ_SPLIT_BF16X3, "emu": cq.CQ_FP64_EMU}[args.prec]
    kinds = [k.strip() for k in args.products.split(",") if k.strip()]
    cell = I.diamond_cell(args.ncell, a=WORKLOAD["a_bohr"], sigma=WORKLOAD["sigma_bohr"],
                          seed=WORKLOAD["seed"], norb=9)
    ctx = cq.Context(dev)
    t = lambda a, dt: torch.tensor(a, dtype=dt, device=f"cuda:{dev}")
    pos, nb = t(cell.pos, torch.float64), t(cell.nb, torch.int32)
    radii = sorted({WORKLOAD[r] for k in kinds for r in PRODUCTS[k]})
    pats = {r: ctx.pattern(pos, cell.box, nb, r) for r in radii}
    vals = {}
    for k in kinds:
        for r in PRODUCTS[k][:2]:
            rr = WORKLOAD[r]
            if rr not in vals:
                pb = I.random_blocks(cell, rr, int(rr), symmetric=False)
                vals[rr] = ctx.scatter(pats[rr], t(pb.i, torch.int32), t(pb.j, torch.int32),
                                       t(pb.off, torch.int64), t(pb.values, torch.float64))
    out = {"mode": "products", "workload": workload_name(cell.n_atoms), "prec": args.prec,
           "steps": args.steps}
    for k in kinds:
        ra, rb, rc = (WORKLOAD[r] for r in PRODUCTS[k])
        C = ctx.zeros(pats[rc])
        ctx.bsmm(1.0, pats[ra], vals[ra], pats[rb], vals[rb], 0.0, pats[rc], C, prec=prec)
        ctx.sync()
        ctx.set_timing(True)
        ctx.kernel_stats()
        for _ in range(args.steps):
            ctx.bsmm(1.0, pats[ra], vals[ra], pats[rb], vals[rb], 0.0, pats[rc], C, prec=prec)
        n, ms, fl, mma = ctx.kernel_stats()
        ctx.set_timing(False)
        out[k] = {"kernel_ms": ms / args.steps, "launches": n,
                  "useful_tflops": fl / (ms * 1e-3) / 1e12 if ms else None,
                  "issued_tflops": mma / (ms * 1e-3) / 1e12 if ms and mma else None}
        del C
        if prec != cq.CQ_FP64:
            ctx.release_cache()  # the next kind's plan and pieces start from free memory
    print(json.dumps(out), flush=True)
    ctx.close()


def main():
    args = parse()
    if args.sweep:
        run_sweep(args, int(os.environ.get("LOCAL_RANK", 0)))
        return
    if args.converge:
        run_converge(args, int(os.environ.get("LOCAL_RANK", 0)))
        return
    if args.solvers:
        run_solvers(args, int(os.environ.get("LOCAL_RANK", 0)))
        return
    if args.products:
        run_products(args, int(os.environ.get("LOCAL_RANK", 0)))
        return
    if args.batch_c4:
        run_batch_c4(args, int(os.environ.get("LOCAL_RANK", 0)))
        return
    if args.converge_emu:
        run_converge_emu(args, int(os.environ.get("LOCAL_RANK", 0)))
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_cq(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
