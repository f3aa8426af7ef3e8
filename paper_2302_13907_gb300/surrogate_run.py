"""Train the trace surrogate on simulator traces, gate it, fall back to the
simulator, and report accuracy and throughput against the plain solver.

    python -m paper_2302_13907_gb300.surrogate_run --train train.npz --test test.npz \
        --out report.json [--params params.npz] [--epochs 400]

train/test .npz come from `surrogate_data` (X [n][6] case parameters,
Y [n][8][2048] reflected-window traces, seeds, sim_seconds).  Every step of
training and inference runs in the library's kernels; the simulator runs the
cases the gate rejects.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import workloads as W
from .binding import BatchSimulation, Surrogate

TOL = 0.05  # relative L2 error a surrogate answer may have


def rel_err(pred, true):
    d = (pred - true).reshape(len(true), -1)
    t = true.reshape(len(true), -1)
    return np.linalg.norm(d, axis=1) / np.linalg.norm(t, axis=1)


def simulate(seeds, stream=None):
    """Reflected-window traces of the given cases by the batched simulator; wall seconds."""
    from .surrogate_data import WINDOW

    if len(seeds) == 0:
        return np.zeros((0, 8, WINDOW), np.float32), 0.0
    t0 = time.perf_counter()
    out = []
    for b0 in range(0, len(seeds), 64):
        cases = [W.scenario_case(int(s), surrogate_inputs=True) for s in seeds[b0:b0 + 64]]
        steps = cases[0].steps
        with BatchSimulation(cases, graph_chunk=100, stream=stream, max_steps=steps) as B:
            B.run(steps)
            B.sync()
            out += [B.traces(c)[:, steps - WINDOW:] for c in range(len(cases))]
    return np.asarray(out, np.float32), time.perf_counter() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", required=True)
    ap.add_argument("--test", required=True)
    ap.add_argument("--out", required=True)
    ap.add_argument("--params", default=None)
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--val-frac", type=float, default=0.15)
    ap.add_argument("--k", type=int, default=3)
    ap.add_argument("--gate-margin", type=float, default=1.0,
                    help="accept a case only where its nearest validation cases are within margin * 5 %%")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--fallback", action="store_true", help="run the simulator on the rejected test cases")
    a = ap.parse_args()

    tr = np.load(a.train)
    te = np.load(a.test)
    X, Y = tr["X"].astype(np.float32), tr["Y"].astype(np.float32)
    Xt, Yt = te["X"].astype(np.float32), te["Y"].astype(np.float32)
    rng = np.random.default_rng(a.seed)
    perm = rng.permutation(len(X))
    nv = max(1, int(round(a.val_frac * len(X))))
    iv, it = perm[:nv], perm[nv:]
    x_mean = X[it].mean(axis=0)
    x_scale = np.maximum(X[it].std(axis=0), 1e-12)
    y_scale = float(np.sqrt(np.mean(Y[it].astype(np.float64) ** 2)))

    S = Surrogate(max_batch=64, seed=a.seed + 1)
    S.set_normalization(x_mean, x_scale, y_scale)
    t0 = time.perf_counter()
    hist = S.train(X[it], Y[it], epochs=a.epochs, batch=a.batch, lr=a.lr, seed=a.seed)
    t_train = time.perf_counter() - t0

    e_val = rel_err(S.forward(X[iv]), Y[iv])
    S.gate_fit(X[iv], e_val)
    S.forward(Xt[:4])  # warm
    t0 = time.perf_counter()
    P = S.forward(Xt)
    t_inf = time.perf_counter() - t0
    e_test = rel_err(P, Yt)
    acc = S.gate(Xt, k=a.k, tol=TOL * a.gate_margin)

    t_sim_plain = float(te["sim_seconds"]) if "sim_seconds" in te.files else None
    per_case_sim = t_sim_plain / len(Xt) if t_sim_plain else None
    rejected = np.flatnonzero(~acc)
    t_fallback = None
    if a.fallback and len(rejected):
        Yf, t_fallback = simulate(te["seeds"][rejected])
        P[rejected] = Yf
    elif per_case_sim is not None:
        t_fallback = per_case_sim * len(rejected)
    final_err = rel_err(P, Yt)
    n = len(Xt)
    rep = {
        "train_cases": int(len(it)), "val_cases": int(nv), "test_cases": int(n), "params": int(S.n_params),
        "epochs": a.epochs, "train_seconds": t_train, "loss_first": float(hist[0]), "loss_last": float(hist[-1]),
        "val_rel_l2_median": float(np.median(e_val)),
        "test_rel_l2_median": float(np.median(e_test)), "test_rel_l2_p90": float(np.quantile(e_test, 0.9)),
        "test_frac_within_5pct": float(np.mean(e_test <= TOL)),
        "gate_k": a.k, "gate_tol": TOL * a.gate_margin, "gate_accept_frac": float(acc.mean()),
        "gate_accepted_within_5pct": float(np.mean(e_test[acc] <= TOL)) if acc.any() else None,
        "final_frac_within_5pct": float(np.mean(final_err <= TOL + 1e-7)),
        "inference_seconds": t_inf, "surrogate_cases_per_s": n / t_inf,
        "plain_solver_seconds": t_sim_plain, "plain_cases_per_s": (n / t_sim_plain) if t_sim_plain else None,
        "fallback_cases": int(len(rejected)), "fallback_seconds": t_fallback,
        "fallback_measured": bool(a.fallback and len(rejected)),
    }
    if t_sim_plain and t_fallback is not None:
        tot = t_inf + t_fallback
        rep["surrogate_plus_fallback_cases_per_s"] = n / tot
        rep["speedup_vs_plain"] = t_sim_plain / tot
    rep["epoch_loss"] = [float(x) for x in hist[:: max(1, len(hist) // 50)]]
    json.dump(rep, open(a.out, "w"), indent=1)
    if a.params:
        np.savez_compressed(a.params, theta=S.params(), x_mean=x_mean, x_scale=x_scale, y_scale=y_scale)
    print(json.dumps({k: v for k, v in rep.items() if k != "epoch_loss"}, indent=1))


if __name__ == "__main__":
    main()
