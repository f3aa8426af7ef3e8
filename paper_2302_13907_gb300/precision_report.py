"""Storage-precision report: FP32 / BF16 / FP16 / FP16 with stochastic
rounding storage of the fields (FP32 arithmetic, FP64 trace accumulation).

    python -m paper_2302_13907_gb300.precision_report --crop-ref REF.npz --out report.json [--full]

* crop: the Nz = 1024 crop (z in [8.0, 10.56) m) of the 20 m well, 20000 steps,
  per-receiver relative L2 and max-abs error of each storage type against the
  FP64 oracle traces stored in REF.npz (written by
  tests/golden/make_crop_reference.py) and against the FP32 GPU run;
* full (--full): the 20 m well, 20000 steps, each storage type against FP32.
Throughput (Gcell-updates/s) of each run is reported beside its error.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import workloads as W
from .binding import Simulation


def errors(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    per = []
    for q in range(ref.shape[0]):
        nr = np.linalg.norm(ref[q])
        per.append({"rel_l2": float(np.linalg.norm(got[q] - ref[q]) / nr) if nr > 0 else None,
                    "max_abs": float(np.abs(got[q] - ref[q]).max()), "ref_peak": float(np.abs(ref[q]).max())})
    allrel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    return {"rel_l2_all": allrel, "per_receiver": per}


def run(sc, storage, steps, stream=None):
    import torch

    with Simulation(sc, storage=storage, max_steps=steps, graph_chunk=200, stream=stream) as s:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(steps)
        s.sync()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        tr = s.traces()
        kind, tile = s.config()
    return tr, sc.grid.cells * steps / dt / 1e9, kind, tile


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--crop-ref", required=True)
    ap.add_argument("--out", required=True)
    ap.add_argument("--full", action="store_true")
    ap.add_argument("--steps", type=int, default=20000)
    a = ap.parse_args()
    import torch

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ref = np.load(a.crop_ref)
    rep = {"crop": {}, "full": {}}
    full = W.config2()
    crop = W.config3_crop(full)
    steps = min(a.steps, int(ref["steps"]))
    oracle_tr = ref["traces"][:, :steps]
    f32 = None
    for st in ("f32", "bf16", "f16", "f16sr"):
        tr, rate, kind, tile = run(crop, st, steps, stream.cuda_stream)
        e = {"vs_oracle_fp64": errors(tr, oracle_tr), "gcell_updates_per_s": rate, "kernel": kind, "tile": tile}
        if f32 is None:
            f32 = tr
        else:
            e["vs_gpu_fp32"] = errors(tr, f32)
        rep["crop"][st] = e
        print(st, "crop rel-L2 vs FP64", e["vs_oracle_fp64"]["rel_l2_all"], flush=True)
    rep["crop"]["workload"] = f"{crop.name}, {steps} steps, receivers at z = 8.0, 8.5, 9.0, 9.5 m"
    if a.full:
        f32 = None
        for st in ("f32", "bf16", "f16", "f16sr"):
            tr, rate, kind, tile = run(full, st, a.steps, stream.cuda_stream)
            e = {"gcell_updates_per_s": rate, "kernel": kind, "tile": tile}
            if f32 is None:
                f32 = tr
            else:
                e["vs_gpu_fp32"] = errors(tr, f32)
            rep["full"][st] = e
            print(st, "full", e.get("vs_gpu_fp32", {}).get("rel_l2_all"), rate, flush=True)
        rep["full"]["workload"] = f"{full.name}, {a.steps} steps, 16 receivers"
    json.dump(rep, open(a.out, "w"), indent=1)


if __name__ == "__main__":
    main()
