"""Training / test data of the trace surrogate, generated by the simulator.

Each sample is one cement-hardening case (136 x 32 x Nz cylindrical grid,
uneven Nz, FP32, 6000 steps) run in batches of up to 64 wells per launch;
the target is the last 2048 steps (the reflected window) of the 8 axis
receivers, the input the six case parameters (cement-top depth, ramp
length, top shear fraction, casing thickness, cement Vs, rock Vs).

    python -m paper_2302_13907_gb300.surrogate_data --out data.npz \
        --seeds 1000:1320 [--batch 64]
"""
from __future__ import annotations

import argparse
import time

import numpy as np

from . import workloads as W

WINDOW = 2048


def parse_seeds(spec: str):
    out = []
    for part in spec.split(","):
        if ":" in part:
            a, b = part.split(":")
            out.extend(range(int(a), int(b)))
        else:
            out.append(int(part))
    return out


def generate(seeds, batch=64, stream=None, log=print):
    from .binding import BatchSimulation

    X, Y = [], []
    t0 = time.time()
    for b0 in range(0, len(seeds), batch):
        chunk = seeds[b0:b0 + batch]
        cases = [W.scenario_case(s, surrogate_inputs=True) for s in chunk]
        steps = cases[0].steps
        with BatchSimulation(cases, graph_chunk=100, stream=stream, max_steps=steps) as B:
            B.run(steps)
            B.sync()
            for c, sc in enumerate(cases):
                tr = B.traces(c)
                Y.append(tr[:, steps - WINDOW:])
                X.append(W.surrogate_features(sc))
        log(f"{b0 + len(chunk)}/{len(seeds)} cases, {time.time() - t0:.0f} s")
    return np.asarray(X, np.float64), np.asarray(Y, np.float32), time.time() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--seeds", required=True)
    ap.add_argument("--batch", type=int, default=64)
    a = ap.parse_args()
    seeds = parse_seeds(a.seeds)
    X, Y, secs = generate(seeds, a.batch)
    np.savez_compressed(a.out, X=X, Y=Y, seeds=np.asarray(seeds), sim_seconds=secs)
    print("wrote", a.out, X.shape, Y.shape)


if __name__ == "__main__":
    main()
