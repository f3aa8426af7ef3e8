"""Write the FP64 oracle's receiver traces on the Nz = 1024 crop of the 20 m
well (z in [8.0, 10.56) m, same rock noise), the reference of the storage
precision report.  Calls only the oracle and the seeded workload generator.

    python tests/golden/make_crop_reference.py [--steps 20000] [--threads N]

Output: tests/golden/crop1024_oracle_traces.npz with the traces [4][steps]
(float64), dt, and a SHA-256 of the medium (cell IDs and table) so a user can
check that the generator reproduced the same medium.
"""
import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2302_13907_gb300 import workloads as W  # noqa: E402


def medium_hash(med) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(med.cell_id).tobytes())
    for a in (med.rho, med.vp, med.vs):
        h.update(np.ascontiguousarray(a, np.float64).tobytes())
    return h.hexdigest()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--out", default=os.path.join(HERE, "crop1024_oracle_traces.npz"))
    a = ap.parse_args()
    sc = W.config3_crop()
    o = oracle.Oracle(sc, max_steps=a.steps, threads=a.threads)
    t0 = time.time()
    done = 0
    while done < a.steps:
        n = min(500, a.steps - done)
        o.step(n)
        done += n
        print(f"{done}/{a.steps} steps, {time.time() - t0:.0f} s", flush=True)
    np.savez_compressed(a.out, traces=o.traces(), dt=o.dt, steps=a.steps, medium_sha256=medium_hash(sc.medium),
                        receivers_z=sc.receivers.z, name=sc.name)
    print("wrote", a.out)


if __name__ == "__main__":
    main()
