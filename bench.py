"""Benchmark of the cased-well simulator on the 20 m full-scale well.

Workload: Nr = 180 (dr 2.5 mm) + 16 PML cells, Ntheta = 64, Nz = 8192
(dz 2.5 mm) + 2 x 16 PML cells = 64 x 196 x 8224 = 103,161,856 cells, FP32, graded cement top,
correlated rock noise, 8 kHz axis monopole, 16 axis receivers.  One bench
step = `--chunk` leapfrog steps (one CUDA-graph replay) of the whole grid;
the metric is cell-updates per second including PML cells.  The state
(3.7 GB of fields) is far larger than L2, so no flush is needed between
steps.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
Under torchrun every rank runs an independent replica on its own GPU
(the single-well problem does not shard without a halo exchange) and
rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s"
L2_BYTES = 129 * 2 ** 20


def shard(n, rank, ws):
    """Units (cases) rank `rank` of `ws` takes: round robin, so every rank's
    share has the same mix of sizes.  No data-path collective is needed."""
    return list(range(rank, n, ws))


def max_over_ranks(x, pg, device="cuda"):
    """The largest x over all ranks (the whole job's time); x without a group."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, pg, device="cuda"):
    """The sum of x over all ranks (the whole job's units); x without a group."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# GB300's nominal HBM3e bandwidth (the chip's data-sheet figure); the measured
# copy bandwidth above is the roofline's denominator, this one a second ceiling
SPEC_HBM_GBS = 7900.0


def kernel_hash() -> str:
    """Hash of the uniform-grid stencil sources and the device headers they
    include (the kernels the stored DRAM traffic was captured on; the refined
    grid's interface kernel is not one, nor is the host-side state header),
    comments and blank space removed, so that only a change of code voids it."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2302_13907_gb300", "csrc")
    files = glob.glob(os.path.join(csrc, "stencil_*.cu")) + [os.path.join(csrc, "cwell_internal.cuh"),
                                                             os.path.join(csrc, "tma_util.cuh"),
                                                             os.path.join(csrc, "hoist_body.cuh")]
    for f in sorted(f for f in files if os.path.basename(f) != "stencil_refine.cu"):
        code = re.sub(r"/\*.*?\*/", " ", open(f).read(), flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [l.strip().split(",") for l in open(self.f.name) if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def split_half_code(tile, vel):
    """Split code of one half: a pair code v * 10000 + s runs v's velocity
    kernel and s's stress kernel."""
    return (tile // 10000 if vel else tile % 10000) if tile >= 10000 else tile


def split_kernel_name(tile, vel):
    """Name of one half of the split path, with its split code: 'vel:2205'.
    2000 = plain split kernels, 20xx / 21xx = load-first kernels, 22xx =
    interior + edge launches (one half = both launches)."""
    return f"{'vel' if vel else 'str'}:{split_half_code(tile, vel)}"


def launches_per_step(kind, tile):
    """Kernel launches of one leapfrog step (volumetric source): the fused
    kernel or the two halves, plus the receiver kernel; an interior / edge
    split half (22xx) is two launches, a three-way split half (23xx) three."""
    if kind in (2, 5):  # fused or sweep kernel + receivers
        return 2
    if kind == 4:
        return 3
    per_half = {22: 2, 23: 3}  # interior + edge; interior + radial + ends
    return 1 + sum(per_half.get(split_half_code(tile, v) // 100, 1) for v in (True, False))


def kernel_label(kind, tile):
    """Name of the path sim_config reports (kernel kind, tile code)."""
    if kind == 2:
        return "fused4" if tile >= 100 else "fused"
    if kind == 4:
        return "march"
    if kind == 5:
        return f"sweep ({tile})"
    if tile >= 10000:
        return f"split (velocity {split_half_code(tile, True)}, stress {split_half_code(tile, False)})"
    return "split (load-first)" if tile > 2000 else "split"


def alg_bytes_split(g, elem=4):
    """Algorithmic bytes per cell-update of the split kernels: each field read
    once and written once where updated, the material ID read once, PML memory
    variables read and written in their slabs."""
    cells = g.nth * g.NR * g.NZ
    fr = g.pml_r / g.NR
    fz = 2 * g.pml_z / g.NZ
    vel = 9 * elem + 2 + 3 * elem + fr * 6 * 8 + fz * 3 * 8
    strs = 9 * elem + 2 + 6 * elem + fr * 6 * 8 + fz * 3 * 8
    return cells, vel, strs


def alg_bytes_fused(g, elem=4):
    """Algorithmic bytes per cell-update of the fused kernel: all nine fields
    read once and written once, the material ID read once, every PML memory
    variable read and written once in its slab."""
    fr = g.pml_r / g.NR
    fz = 2 * g.pml_z / g.NZ
    return 18 * elem + 2 + fr * 12 * 8 + fz * 6 * 8


def cpu_sample(sc, seconds=15.0, nz=128):
    """Oracle on a bounded sample of the workload: the full radius and azimuth
    of the well, `nz` interior cells around the source, as many steps as fit
    in ~`seconds` of host time."""
    import oracle
    from paper_2302_13907_gb300 import workloads as W

    g = sc.grid
    ks = int(round(sc.source.z / g.dz))
    k0 = max(0, ks - nz // 2)
    crop = W.crop_z(sc.medium, k0, nz)
    sub = W.Scenario("sample", crop, W.Source(z=sc.source.z - k0 * g.dz, f0=sc.source.f0),
                     W.on_axis_receivers([sc.source.z - k0 * g.dz]), cfl=sc.cfl, steps=100000)
    o = oracle.Oracle(sub, max_steps=100000)
    t0 = time.perf_counter()
    o.step(5)
    t1 = time.perf_counter()
    n = max(5, int(seconds / max((t1 - t0) / 5, 1e-6)))
    t0 = time.perf_counter()
    o.step(n)
    t1 = time.perf_counter()
    cells = crop.grid.nth * crop.grid.NR * crop.grid.NZ
    return dict(value=cells * n / (t1 - t0) / 1e9, unit=METRIC, cores=oracle.max_threads(), kind="oracle",
                sample=f"FP64 oracle, {crop.grid.nth}x{crop.grid.NR}x{crop.grid.NZ} z-crop around the source "
                       f"({cells} cells), {n} steps, {t1 - t0:.1f} s"), (cells, o)


def bench_batch(stream, n_cases=64, steps=60, warm=8, rank=0, ws=1, pg=None):
    """Batched scenarios (the 64 cement-hardening cases, uneven Nz) in one
    persistent launch per kernel per step, against the same cases run one
    after another with the single-well path.  Throughput is reported in full
    6000-step scenarios per second, measured over `steps` steps.  Under
    torchrun the cases are sharded round robin over the ranks (weak in
    cases per rank, no collective on the data path); times are the max over
    ranks."""
    import torch
    from paper_2302_13907_gb300 import workloads as W
    from paper_2302_13907_gb300.binding import BatchSimulation, Simulation

    cases = [W.scenario_case(s + 1) for s in shard(n_cases, rank, ws)]
    cells = sum_over_ranks(sum(c.grid.cells for c in cases), pg)
    full = cases[0].steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_batch(tile):
        b = BatchSimulation(cases, graph_chunk=steps // 2, stream=stream.cuda_stream, max_steps=steps + warm,
                            tile=tile)
        cfg, lay = b.config(), b.layout()
        b.run(warm)
        torch.cuda.synchronize()
        e0.record(stream)
        b.run(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        b.sync()
        t = e0.elapsed_time(e1) / 1e3
        b.close()
        return t, cfg, lay

    # the batch as built: cases that fill the GPU on their own launches
    # (spread over parallel graph branches), small ones in the shared launches
    tb, (_, items, grid), (own_cases, branches) = timed_batch(0)
    # every case forced into the shared persistent launches
    ts, (_, items_s, grid_s), _ = timed_batch(1)
    tp = 0.0
    for sc in cases:
        s = Simulation(sc, graph_chunk=steps // 2, stream=stream.cuda_stream, max_steps=steps + warm)
        s.step(warm)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        tp += e0.elapsed_time(e1) / 1e3
        s.close()
    tb, tp, ts = max_over_ranks(tb, pg), max_over_ranks(tp, pg), max_over_ranks(ts, pg)
    return {"metric": "scenarios/s", "value": n_cases * steps / full / tb, "plain": n_cases * steps / full / tp,
            "speedup_vs_plain": tp / tb, "gcell_updates_per_s": cells * steps / tb / 1e9,
            "plain_gcell_updates_per_s": cells * steps / tp / 1e9, "cases": n_cases, "cells": cells,
            "steps_timed": steps, "steps_per_scenario": full, "work_items": items, "persistent_blocks": grid,
            "own_launch_cases": own_cases, "branches": branches,
            "path": "every case fills the GPU (>= 4 Mi cells): each runs its own tuned split launches, the cases "
                    f"spread over {branches} parallel graph branches",
            "all_shared": {"value": n_cases * steps / full / ts, "speedup_vs_plain": tp / ts,
                           "work_items": items_s, "persistent_blocks": grid_s,
                           "path": "every case forced into the shared persistent work-list launches"},
            "error": "each batched case equals its single run (rel-L2 <= 1e-6, tested); FP32 vs FP64 oracle <= 1e-4",
            "workload": "64 cement-hardening cases: 136 x 32 x Nz, Nz in {2080, 3104, 4128, 6176} with PML, FP32",
            "sharding": f"cases round robin over {ws} rank(s)"}


def bench_batch_small(stream, n_cases=64, steps=400, warm=8, rank=0, ws=1, pg=None):
    """The batching machinery on small wells, where one case cannot fill the
    GPU: 64 miniature cement cases (44 x 8 x 256 cells each) batched against
    the same cases run one after another; full 1200-step scenarios per second
    (cases sharded over the ranks as bench_batch)."""
    import torch
    from paper_2302_13907_gb300 import workloads as W
    from paper_2302_13907_gb300.binding import BatchSimulation, Simulation

    cases = [W.small_cement_case(s) for s in shard(n_cases, rank, ws)]
    full = cases[0].steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with BatchSimulation(cases, graph_chunk=steps // 2, stream=stream.cuda_stream, max_steps=steps + warm) as b:
        b.run(warm)
        torch.cuda.synchronize()
        e0.record(stream)
        b.run(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        tb = e0.elapsed_time(e1) / 1e3
    tp = 0.0
    for sc in cases:
        with Simulation(sc, graph_chunk=steps // 2, stream=stream.cuda_stream, max_steps=steps + warm) as s:
            s.step(warm)
            torch.cuda.synchronize()
            e0.record(stream)
            s.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            tp += e0.elapsed_time(e1) / 1e3
    tb, tp = max_over_ranks(tb, pg), max_over_ranks(tp, pg)
    return {"metric": "scenarios/s", "value": n_cases * steps / full / tb, "plain": n_cases * steps / full / tp,
            "speedup_vs_plain": tp / tb, "cases": n_cases, "steps_timed": steps, "steps_per_scenario": full,
            "workload": "64 miniature cement cases: 44 x 8 x 256 cells with PML, FP32"}


def bench_refined(stream, sc, uniform_value, uniform_dt, steps=400, warm=20, tile=0):
    """The same well on the azimuthally refined grid (zones by the paper's
    rule, Sec. 3: 4 / 8 / 16 / 32 / 64 azimuthal nodes from the axis out):
    cell-update throughput, and the physical time simulated per wall-clock
    second against the uniform grid's (the coarse zones near the axis let
    the CFL step grow and hold fewer cells)."""
    import torch
    from paper_2302_13907_gb300 import workloads as W
    from paper_2302_13907_gb300.binding import RefinedSimulation

    g = sc.grid
    rows = W.refinement_rows(g)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with RefinedSimulation(sc, rows, graph_chunk=steps // 2, stream=stream.cuda_stream, max_steps=steps + warm,
                           tile=tile) as r:
        r.step(warm)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()  # a second profiler range: the refined grid's timed steps
        e0.record(stream)
        r.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        t = e0.elapsed_time(e1) / 1e3
        r.sync()
        cells, dt, zones = r.cells, r.dt, r.zones
    uniform_cells = g.nth * g.NR * g.NZ
    sim_us = dt * steps / t * 1e6
    uni_us = uniform_dt * uniform_value * 1e9 / uniform_cells * 1e6
    return {"metric": "simulated us per s", "value": sim_us, "uniform": uni_us, "speedup_vs_uniform": sim_us / uni_us,
            "gcell_updates_per_s": cells * steps / t / 1e9, "cells_per_step": cells,
            "uniform_cells_per_step": uniform_cells, "dt": dt, "uniform_dt": uniform_dt,
            "zones": [{"first_row": a, "rows": b, "nth": c} for a, b, c in zones], "steps_timed": steps,
            "split_codes": tile or 22852324,
            "error": "GPU vs the refined FP64 oracle: fields <= 2e-5 of scale, traces <= 1e-4 rel-L2 (tested)"}


SURROGATE_PARAMS = os.path.join(ROOT, "paper_2302_13907_gb300", "data", "surrogate_cement.npz")


def bench_surrogate(stream, n_check=8, n_plain=2):
    """The trace surrogate on its 512 held-out cement cases (seeds 9000 ..
    9511): inference of all cases, the gate (nearest validation errors and
    the network's sensitivity), the simulator on every
    rejected case (the fallback: the refined-grid simulator on the case's
    reach crop, which generated the training data), timed together as cases/s;
    against the plain FP32 solver (uniform grid, whole well, 6000 steps),
    timed on a sample of `n_plain` cases and extrapolated to all.  The
    accuracy of accepted answers is checked live on `n_check` of them; the
    full-set figures come from the committed training report."""
    import torch
    from paper_2302_13907_gb300 import surrogate_data as D
    from paper_2302_13907_gb300 import surrogate_run as R
    from paper_2302_13907_gb300 import workloads as W
    from paper_2302_13907_gb300.binding import SURROGATE_DEFAULT, Simulation, Surrogate

    if not os.path.exists(SURROGATE_PARAMS):
        return {"unavailable": "trained parameters not in the repository"}
    d = np.load(SURROGATE_PARAMS)
    seeds = [int(x) for x in d["test_seeds"]]
    k, margin = int(d["gate_k"]), float(d["gate_margin"])
    S = Surrogate(max_batch=64, seed=1, stream=stream.cuda_stream)
    S.set_params(R.unpack_params(d["w_bf16"], d["biases"], SURROGATE_DEFAULT))
    S.set_normalization(d["x_mean"], d["x_scale"], float(d["y_scale"]))
    S.gate_fit(d["gate_x"], d["gate_err"])
    Xt = np.stack([W.case_features(sd) for sd in seeds]).astype(np.float32)
    S.forward(Xt[:4])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P = S.forward(Xt)
    acc = R.gate_decision(S, Xt, d)  # the neighbour rule and, when saved, the sensitivity bound
    t_inf = time.perf_counter() - t0
    rejected = np.flatnonzero(~acc)
    t0 = time.perf_counter()
    if len(rejected):  # the fallback on every rejected case, several cases in flight
        _, Yf, _ = D.generate_refined([seeds[q] for q in rejected], log=lambda m: None)
        P[rejected] = Yf
    torch.cuda.synchronize()
    t_fb = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    chk = rng.choice(np.flatnonzero(acc), size=min(n_check, int(acc.sum())), replace=False)
    errs, t_fallback = [], []
    if len(chk):
        t0 = time.perf_counter()
        _, Yc, _ = D.generate_refined([seeds[q] for q in chk], log=lambda m: None)
        t_fallback = [(time.perf_counter() - t0) / len(chk)]
        errs = [float(x) for x in R.rel_err(P[chk], Yc)]
    t_plain = []
    for sd in seeds[:n_plain]:
        sc = W.scenario_case(sd, surrogate_inputs=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with Simulation(sc, graph_chunk=200, stream=stream.cuda_stream, max_steps=sc.steps) as s:
            s.step(sc.steps)
            s.sync()
        t_plain.append(time.perf_counter() - t0)
    n = len(seeds)
    tot = t_inf + t_fb
    rep_path = os.path.join(ROOT, "profiles", "surrogate_cement_report.json")
    full = json.load(open(rep_path)) if os.path.exists(rep_path) else {}
    return {"metric": "cases/s", "cases_per_s": n / tot, "cases": n, "accepted_frac": float(acc.mean()),
            "fallback_cases": int(len(rejected)), "inference_and_gate_s": t_inf, "fallback_s": t_fb,
            "plain_cases_per_s": 1.0 / float(np.mean(t_plain)), "plain_sample": len(t_plain),
            "speedup_vs_plain": float(np.mean(t_plain)) * n / tot,
            "fallback_cases_per_s": 1.0 / float(np.mean(t_fallback)) if t_fallback else None,
            "speedup_vs_fallback": float(np.mean(t_fallback)) * n / tot if t_fallback else None,
            "fallback": "refined grid on each case's 1.6 m reach crop, several cases in flight",
            "max_accepted_rel_l2_sampled": max(errs) if errs else None, "accepted_checked": len(errs),
            "max_accepted_rel_l2": full.get("max_accepted_rel_l2"),
            "false_accepts": full.get("false_accepts"), "gate_margin": margin, "gate_k": k,
            "gate_sens_max": float(d["gate_sens_max"]) if "gate_sens_max" in d.files else None,
            "tolerance": R.TOL,
            "workload": "512 held-out cement cases (seeds 9000-9511); inputs: top depth, ramp, top shear fraction, "
                        "casing thickness, cement Vs, rock Vs; output 8 x 2048 reflected-window traces",
            "note": "max_accepted_rel_l2 and false_accepts: all 512 cases, from the surrogate job's report"}


def run_reference(args, ws, rank):
    """--impl reference: the FP64 CPU oracle on bounded samples of the same workload."""
    if rank != 0:
        return
    from paper_2302_13907_gb300 import workloads as W
    import oracle

    sc = W.config2()
    g = sc.grid
    ks = int(round(sc.source.z / g.dz))
    nz = 128
    k0 = max(0, ks - nz // 2)
    crop = W.crop_z(sc.medium, k0, nz)
    sub = W.Scenario("sample", crop, W.Source(z=sc.source.z - k0 * g.dz, f0=sc.source.f0),
                     W.on_axis_receivers([sc.source.z - k0 * g.dz]), cfl=sc.cfl, steps=100000)
    o = oracle.Oracle(sub, max_steps=100000)
    cells = crop.grid.nth * crop.grid.NR * crop.grid.NZ
    per = 10  # leapfrog steps per bench step
    for _ in range(args.warmup):
        o.step(per)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(per)
    dt = time.perf_counter() - t0
    v = cells * per * args.steps / dt / 1e9
    line = {"metric": METRIC, "value": v, "unit": METRIC, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": sc.name + " (bounded z-crop sample around the source, FP64 oracle)",
                       "sample_cells": cells, "steps_per_bench_step": per},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"{crop.grid.nth}x{crop.grid.NR}x{crop.grid.NZ} crop, {per} steps per bench step"},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--chunk", type=int, default=200, help="leapfrog steps per bench step")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16", "f16sr"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "split", "fused", "fused4", "march", "sweep"])
    ap.add_argument("--tile", type=int, default=0, help="tile code to force (0: the autotuner picks)")
    ap.add_argument("--refined-tile", type=int, default=0,
                    help="split code (or pair) of the refined grid's zones (0: the library's choice by size)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--nz", type=int, default=8192, help="interior z cells (8192 = the 20 m well; smaller for profiling)")
    ap.add_argument("--nr", type=int, default=180, help="interior radial cells (180 = the 20 m well; smaller for profiling)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-scenarios measurement")
    ap.add_argument("--no-refined", action="store_true", help="skip the azimuthally refined grid measurement")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the trace-surrogate measurement")
    args = ap.parse_args()
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import torch

    pg = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        pg = dist
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    # a dedicated stream: the library enqueues on it and the CUDA events are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    from paper_2302_13907_gb300 import workloads as W
    from paper_2302_13907_gb300.binding import Simulation

    sc = W.config2(nz=args.nz, nr=args.nr)
    g = sc.grid
    cells = g.nth * g.NR * g.NZ
    K, Wm, T = args.steps, args.warmup, args.chunk
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        if uuid and not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None

    # ---------------- headline: device-resident, graph replays of T steps
    # (the first sim_create of the process: its tuner times every candidate;
    # the e2e figure below reuses the tuner's choice, so this cold cost is
    # reported on its own)
    torch.cuda.synchronize()
    t_cold = time.perf_counter()
    sim = Simulation(sc, storage=args.storage, kernel=args.kernel, tile=args.tile, graph_chunk=T, stream=stream.cuda_stream,
                     max_steps=(K + Wm) * T + 1)
    torch.cuda.synchronize()
    cold_create_s = time.perf_counter() - t_cold
    for _ in range(Wm):
        sim.step(T)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = Clocks(uuid)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    # the profiler range marks the timed region for `ncu --profile-from-start off` (a no-op otherwise)
    torch.cuda.profiler.start()
    e0.record(stream)
    for _ in range(K):
        sim.step(T)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    ck = clocks.stop()
    if pg:
        pg.barrier()
    ms = e0.elapsed_time(e1)
    sim.sync()
    bytes_held = sim.device_bytes
    uniform_dt = sim.dt
    sim.close()
    del sim
    ms = max_over_ranks(ms, pg)
    value = ws * cells * T * K / (ms / 1e3) / 1e9

    # ---------------- roofline: per-kernel CUDA events on the launching stream
    peak, peak_kind = _peaks()
    elem = 4 if args.storage == "f32" else 2
    _, b_vel, b_str = alg_bytes_split(g, elem)
    b_fused = alg_bytes_fused(g, elem)
    tsim = Simulation(sc, storage=args.storage, kernel=args.kernel, tile=args.tile, stream=stream.cuda_stream, timing=True,
                      max_steps=64)
    kind, tile = tsim.config()
    tsim.step(3)
    base = [tsim.kernel_time(q) for q in range(3)]
    tsim.step(30)
    kt = [tsim.kernel_time(q) for q in range(3)]
    tsim.close()
    avg = [(kt[q][0] - base[q][0]) / max(1, kt[q][1] - base[q][1]) for q in range(3)]
    if kind == 2:
        names = ["fused4_step" if tile >= 100 else "fused_step", "-", "receivers"]
        qd, per_cell = 0, b_fused
    elif kind == 5:  # one launch per step: both halves, every field read and written once
        names = [f"sweep_step:{tile}", "-", "receivers"]
        qd, per_cell = 0, b_fused
    else:
        names = ["march_step(velocity)", "march_step(stress)", "receivers"] if kind == 4 else \
            [split_kernel_name(tile, True), split_kernel_name(tile, False), "receivers"]
        qd = 0 if avg[0] >= avg[1] else 1
        per_cell = b_vel if qd == 0 else b_str
    alg = per_cell * cells
    achieved = alg / (avg[qd] / 1e3) / 1e9
    traffic = None
    tj = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tj):
        d = json.load(open(tj))
        ent = d.get("kernels", {}).get(names[qd])
        # captured on the full well: reported for that workload only (a crop has
        # another share of edge cells, so scaling by the cell count would mislead)
        if ent and d.get("kernel_hash") == kernel_hash() and ent.get("cells") == cells:
            traffic = ent["dram_bytes_per_launch"]
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": names[qd], "peak_source": f"{peak_kind} hbm_gbs (copy)",
            "frac_vs_spec": achieved / SPEC_HBM_GBS, "spec_peak": SPEC_HBM_GBS,
            "spec_peak_source": "GB300 HBM3e nominal 7.9 TB/s",
            "alg_bytes_per_cell": per_cell, "tile_rows": tile,
            "kernel_ms": {names[q]: avg[q] for q in range(3) if names[q] != "-"}}

    # ---------------- end to end through the C-ABI with host buffers
    e2e = None
    if not args.no_e2e:
        pinned = torch.empty(sc.medium.cell_id.shape, dtype=torch.int16, pin_memory=True)
        pinned.numpy().view(np.uint16)[...] = sc.medium.cell_id
        med_p = W.Medium(g, pinned.numpy().view(np.uint16), sc.medium.rho, sc.medium.vp, sc.medium.vs)
        sc_p = W.Scenario(sc.name, med_p, sc.source, sc.receivers, sc.cfl, sc.steps)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        t0 = time.perf_counter()
        s2 = Simulation(sc_p, storage=args.storage, kernel=args.kernel, tile=args.tile, graph_chunk=T, stream=stream.cuda_stream,
                        max_steps=K * T)
        for _ in range(K):
            s2.step(T)
        tr = s2.traces()
        s2.close()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        wall = max_over_ranks(wall, pg)
        h2d = sc.medium.cell_id.nbytes + sc.medium.rho.nbytes * 4
        e2e = {"value": ws * cells * T * K / wall / 1e9, "unit": METRIC, "h2d_bytes_per_step": h2d / K,
               "d2h_bytes_per_step": tr.nbytes / K,
               "cold_create_s": cold_create_s,
               "note": "sim_create from pinned host arrays (tuner choice cached by the first create of the "
                       "process; cold_create_s = that first sim_create with an empty tuner cache, timed alone) "
                       "+ K x sim_step + sim_traces + sim_destroy, wall clock"}

    batch = None
    if not args.no_batch:
        batch = bench_batch(stream, rank=rank, ws=ws, pg=pg)
        batch["small_cases"] = bench_batch_small(stream, rank=rank, ws=ws, pg=pg)
    refined = None
    if not args.no_refined and args.storage == "f32" and args.nz == 8192 and args.nr == 180:
        refined = bench_refined(stream, sc, value / ws, uniform_dt, tile=args.refined_tile)
    surrogate = None
    if not args.no_surrogate and rank == 0:
        surrogate = bench_surrogate(stream)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, _ = cpu_sample(sc)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": K, "warmup": Wm,
                "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": args.storage if args.storage != "f32" else "f32", "data": "synthetic",
                "config": {"workload": f"{sc.name}: Nr={g.nr}+16 PML, Ntheta=64, Nz={g.nz}+2x16 PML, dr=dz=2.5 mm, "
                                       f"graded cement top, rock noise, 8 kHz monopole, 16 receivers",
                           "cells": cells, "leapfrog_steps_per_bench_step": T,
                           "kernel": kernel_label(kind, tile),
                           "storage": args.storage, "parallelism": f"replicas x{ws}",
                           "l2": f"inputs larger than L2 ({bytes_held / 1e9:.1f} GB resident)"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "batch": batch, "refined": refined,
                "surrogate": surrogate,
                "gpu_launches": K * T * launches_per_step(kind, tile), "clocks": ck}
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
