"""Train the trace surrogate on simulator traces, gate it, fall back to the
simulator, and report accuracy and throughput against the plain solver.

    python -m paper_2302_13907_gb300.surrogate_run --train train.npz --test test.npz \
        --out report.json [--params params.npz] [--epochs 400]

train/test .npz come from `surrogate_data` (X [n][6] case parameters,
Y [n][8][2048] reflected-window traces, seeds, sim_seconds).  Every step of
training and inference runs in the library's kernels; the simulator runs the
cases the gate rejects.

    python -m paper_2302_13907_gb300.surrogate_run --pipeline --out-dir DIR \
        [--phase all|train|gate|test] [--params P] \
        [--train-seeds 1000:5096] [--test-seeds 9000:9512] [--epochs 400]

runs the job with the refined generator of `surrogate_data`.  Phase "train"
generates the training cases, trains, chooses the gate's margin on the
validation cases alone (leave-one-out) and writes DIR/params.npz (weights as
BF16 bit patterns, biases, normalisation, the gate's validation data and
margin) and DIR/train_report.json; phase "gate" adds the second gate signal
(the network's sensitivity, `choose_gate`, on the validation cases alone) to
the saved params; phase "test" generates the held-out cases, times the plain
solver on a sample of them, runs the saved network and gate, falls back to the
simulator on the rejected cases and writes DIR/report.json; "all" runs the
three in one process.
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


def surrogate_shapes(arch):
    """Parameter layout of the network (the order sur_get_params uses):
    W1, b1, W2, b2, W3, b3, (T_l, t_l) per transposed convolution, Wf, bf."""
    ch = list(arch["chans"])
    s = [("W1", (arch["in_dim"], arch["h1"])), ("b1", (arch["h1"],)), ("W2", (arch["h1"], arch["h2"])),
         ("b2", (arch["h2"],)), ("W3", (arch["h2"], arch["l0"] * ch[0])), ("b3", (arch["l0"] * ch[0],))]
    for i in range(len(ch) - 1):
        s += [(f"T{i}", (ch[i], ch[i + 1], 4)), (f"t{i}", (ch[i + 1],))]
    s += [("Wf", (ch[-1], arch["out_ch"])), ("bf", (arch["out_ch"],))]
    return s


def pack_params(theta, arch):
    """Weights as BF16 bit patterns (round to nearest even; the GEMMs read
    BF16), biases FP32."""
    w, b, o = [], [], 0
    for _, sh in surrogate_shapes(arch):
        n = int(np.prod(sh))
        (w if len(sh) > 1 else b).append(theta[o:o + n])
        o += n
    wv = np.concatenate(w).astype(np.float32).view(np.uint32).astype(np.uint64)
    bits = ((wv + 0x7FFF + ((wv >> 16) & 1)) >> 16).astype(np.uint16)
    return bits, np.concatenate(b).astype(np.float32)


def unpack_params(bits, biases, arch):
    w = (bits.astype(np.uint32) << 16).view(np.float32)
    out, wo, bo = [], 0, 0
    for _, sh in surrogate_shapes(arch):
        n = int(np.prod(sh))
        if len(sh) > 1:
            out.append(w[wo:wo + n])
            wo += n
        else:
            out.append(biases[bo:bo + n])
            bo += n
    return np.concatenate(out).astype(np.float32)


def knn_worst(Xn_query, Xn_ref, err_ref, k, exclude_self=False):
    """Largest error among the k nearest reference inputs of each query
    (Euclidean distance in normalised input space), as the gate computes."""
    d = ((Xn_query[:, None, :] - Xn_ref[None, :, :]) ** 2).sum(-1)
    if exclude_self:
        np.fill_diagonal(d, np.inf)
    nn = np.argsort(d, axis=1)[:, :k]
    return err_ref[nn].max(axis=1)


def choose_margin(Xn_val, e_val, k, tol=TOL):
    """The largest margin m (in steps of 0.05) for which the gate, run leave
    one out on the validation cases, accepts no validation case above tol."""
    worst = knn_worst(Xn_val, Xn_val, e_val, k, exclude_self=True)
    best = 0.0
    for m in np.arange(0.05, 1.0001, 0.05):
        acc = worst <= m * tol
        if np.all(e_val[acc] <= tol):
            best = float(m)
    return best


SENS_STEP = 0.1  # input move (normalised units) of the sensitivity signal


def choose_gate(Xn_val, e_val, s_val, k, tol=TOL):
    """The two-signal gate chosen on the validation cases alone: accept a
    query when the largest error among its k nearest validation cases is at
    most margin x tol (leave one out here) and its sensitivity is at most
    sens_max.  For each margin (steps of 0.05) sens_max is the largest
    validation sensitivity below that of every case above tol the neighbour
    rule lets through (infinite when it lets none through); the pair that
    accepts the most validation cases wins (the smaller margin on a tie).
    Returns (margin, sens_max, accepted fraction); no validation case above
    tol is accepted by construction."""
    worst = knn_worst(Xn_val, Xn_val, e_val, k, exclude_self=True)
    bad = e_val > tol
    best = (0.0, 0.0, 0.0)
    for m in np.arange(0.05, 1.0001, 0.05):
        knn_ok = worst <= m * tol
        through = knn_ok & bad
        if through.any():
            below = s_val[s_val < s_val[through].min()]
            smax = float(below.max()) if below.size else -np.inf
        else:
            smax = np.inf
        acc = float(np.mean(knn_ok & (s_val <= smax)))
        if acc > best[2]:
            best = (round(float(m), 2), smax, acc)
    return best


def load_params(path, arch):
    """A Surrogate holding the saved BF16 weights, normalisation and gate."""
    z = np.load(path)
    S = Surrogate(max_batch=64, seed=0)
    S.set_normalization(z["x_mean"], z["x_scale"], float(z["y_scale"]))
    S.set_params(unpack_params(z["w_bf16"], z["biases"], arch))
    S.gate_fit(z["gate_x"], z["gate_err"])
    return S, z


def gate_decision(S, X, z, margin=None, sens_max=None):
    """The saved gate on queries X: the neighbour rule at the saved margin,
    and, when the saved gate has one, the sensitivity bound."""
    k = int(z["gate_k"])
    margin = float(z["gate_margin"]) if margin is None else margin
    acc = S.gate(X, k=k, tol=TOL * margin)
    if sens_max is None and "gate_sens_max" in z.files:
        sens_max = float(z["gate_sens_max"])
    if sens_max is not None and np.isfinite(sens_max):
        step = float(z["gate_sens_step"]) if "gate_sens_step" in z.files else SENS_STEP
        acc &= S.sensitivity(X, step=step) <= sens_max
    return acc


def pipeline_gate(a, log, params):
    """Add the sensitivity signal to a trained network's gate: the
    sensitivity of every validation case on the device, then choose_gate on
    the validation cases alone; the params file is rewritten with the new
    margin and bound."""
    from .binding import SURROGATE_DEFAULT
    S, z = load_params(params, SURROGATE_DEFAULT)
    Xv, ev = z["gate_x"].astype(np.float32), z["gate_err"].astype(np.float64)
    sv = S.sensitivity(Xv, step=SENS_STEP).astype(np.float64)
    Xn = (Xv - z["x_mean"]) / z["x_scale"]
    margin, smax, acc = choose_gate(Xn, ev, sv, int(z["gate_k"]))
    out = {f: z[f] for f in z.files}
    out.update(gate_margin=np.float64(margin), gate_sens_max=np.float64(smax),
               gate_sens_step=np.float64(SENS_STEP), gate_sens=sv.astype(np.float32),
               gate_margin_knn_only=z["gate_margin"] if "gate_margin_knn_only" not in z.files
               else z["gate_margin_knn_only"])
    np.savez_compressed(params, **out)
    log(f"gate: margin {margin}, sensitivity bound {smax:.4g} (step {SENS_STEP}); "
        f"validation accepted {acc:.3f}; validation sensitivity quantiles "
        f"{np.quantile(sv, [0.5, 0.9, 0.99]).round(4)}")
    return margin, smax


def pipeline_train(a, log):
    """Generate the training cases, train, evaluate the BF16 weights on the
    validation cases, choose the gate's margin on them alone (leave-one-out)
    and save DIR/params.npz and DIR/train_report.json."""
    import os
    from . import surrogate_data as D
    from .binding import SURROGATE_DEFAULT

    tr_seeds = D.parse_seeds(a.train_seeds)
    X, Y, t_gen_tr = D.generate_refined(tr_seeds, log=log)
    log(f"generated {len(X)} training cases in {t_gen_tr:.0f} s")
    X, Y = X.astype(np.float32), Y.astype(np.float32)
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
    log(f"trained {len(it)} cases x {a.epochs} epochs in {t_train:.0f} s, loss {hist[0]:.3g} -> {hist[-1]:.3g}")
    # the deployed weights are the BF16 ones: evaluate with exactly those
    bits, biases = pack_params(S.params(), SURROGATE_DEFAULT)
    S.set_params(unpack_params(bits, biases, SURROGATE_DEFAULT))
    e_val = rel_err(S.forward(X[iv]), Y[iv])
    Xn = lambda x: (x - x_mean) / x_scale
    margin = choose_margin(Xn(X[iv]), e_val, a.k)
    np.savez_compressed(os.path.join(a.out_dir, "params.npz"), w_bf16=bits, biases=biases, x_mean=x_mean,
                        x_scale=x_scale, y_scale=np.float64(y_scale), gate_x=X[iv],
                        gate_err=e_val.astype(np.float32), gate_k=np.int64(a.k), gate_margin=np.float64(margin),
                        train_seeds=np.asarray(tr_seeds), test_seeds=np.asarray(D.parse_seeds(a.test_seeds)),
                        val_index=np.asarray(iv), seed=np.int64(a.seed))
    rep = {
        "train_cases": int(len(it)), "val_cases": int(nv), "params": int(S.n_params),
        "epochs": a.epochs, "batch": a.batch, "lr": a.lr, "train_seconds": t_train,
        "loss_first": float(hist[0]), "loss_last": float(hist[-1]),
        "generate_train_seconds": t_gen_tr, "fallback_seconds_per_case_train": t_gen_tr / len(X),
        "val_rel_l2_median": float(np.median(e_val)), "val_rel_l2_max": float(e_val.max()),
        "gate_k": a.k, "gate_margin": margin,
        "epoch_loss": [float(x) for x in hist[:: max(1, len(hist) // 50)]],
    }
    json.dump(rep, open(os.path.join(a.out_dir, "train_report.json"), "w"), indent=1)
    log(f"validation rel-L2 median {np.median(e_val):.4f}, max {e_val.max():.4f}; gate margin {margin}")
    return rep


def pipeline_test(a, log, params, train_rep):
    """Generate the held-out cases, time the plain solver on a sample of them,
    run the saved surrogate and its gate, fall back to the simulator on the
    rejected cases and write DIR/report.json."""
    import os
    from . import surrogate_data as D
    from .binding import SURROGATE_DEFAULT, Simulation

    te_seeds = D.parse_seeds(a.test_seeds)
    Xt, Yt, t_gen_te = D.generate_refined(te_seeds, log=log)
    log(f"generated {len(Xt)} test cases in {t_gen_te:.0f} s")
    # the plain solver (uniform grid, the whole well, 6000 steps) on a sample of the test cases
    plain_t, plain_err = [], []
    for sd, y_ref in zip(te_seeds[:a.plain_sample], Yt[:a.plain_sample]):
        sc = W.scenario_case(sd, surrogate_inputs=True)
        t0 = time.perf_counter()
        with Simulation(sc, graph_chunk=200, max_steps=sc.steps) as s:
            s.step(sc.steps)
            tr = s.traces()[:, sc.steps - D.WINDOW:]
        plain_t.append(time.perf_counter() - t0)
        plain_err.append(float(np.linalg.norm(y_ref - tr) / np.linalg.norm(tr)))
    Xt, Yt = Xt.astype(np.float32), Yt.astype(np.float32)
    S, z = load_params(params, SURROGATE_DEFAULT)
    k, margin = int(z["gate_k"]), float(z["gate_margin"])
    sens_max = float(z["gate_sens_max"]) if "gate_sens_max" in z.files else None
    S.forward(Xt[:4])
    t0 = time.perf_counter()
    P = S.forward(Xt)
    acc = gate_decision(S, Xt, z)
    t_inf = time.perf_counter() - t0
    e_test = rel_err(P, Yt)
    sens = S.sensitivity(Xt, step=SENS_STEP) if sens_max is not None else None
    # the neighbour rule alone at other margins on the same answers: the
    # trade-off the sensitivity bound removes
    sweep = []
    for m in np.arange(0.1, 1.0001, 0.1):
        am = gate_decision(S, Xt, z, margin=float(m), sens_max=np.inf)
        sweep.append({"margin": round(float(m), 2), "accepted_frac": float(am.mean()),
                      "false_accepts": int(np.sum(am & (e_test > TOL))),
                      "max_accepted_rel_l2": float(e_test[am].max()) if am.any() else None})
    rejected = np.flatnonzero(~acc)
    t0 = time.perf_counter()
    if len(rejected):
        _, Yf, _ = D.generate_refined([te_seeds[q] for q in rejected], log=lambda m: None)
        P[rejected] = Yf
    t_fb = time.perf_counter() - t0
    final = rel_err(P, Yt)
    n = len(Xt)
    per_sim = t_gen_te / n
    per_plain = float(np.mean(plain_t)) if plain_t else None
    rep = {k_: v for k_, v in (train_rep or {}).items() if k_ != "epoch_loss"}
    rep.update({
        "test_cases": n,
        "generator": "refined grid (Sec. 3 zoning) on each case's 1.6 m reach crop, traces at the uniform grid's times",
        "generate_test_seconds": t_gen_te, "fallback_seconds_per_case": per_sim,
        "plain_seconds_per_case": per_plain, "plain_sample": len(plain_t),
        "plain_vs_fallback_rel_l2": plain_err,
        "test_rel_l2_median": float(np.median(e_test)), "test_rel_l2_p90": float(np.quantile(e_test, 0.9)),
        "test_rel_l2_max": float(e_test.max()), "test_frac_within_5pct": float(np.mean(e_test <= TOL)),
        "gate_k": k, "gate_margin": margin, "gate_tol": TOL * margin,
        "gate_sens_max": sens_max, "gate_sens_step": SENS_STEP if sens_max is not None else None,
        "test_sens": [round(float(x), 5) for x in sens] if sens is not None else None,
        "accepted": int(acc.sum()), "accepted_frac": float(acc.mean()),
        "max_accepted_rel_l2": float(e_test[acc].max()) if acc.any() else None,
        "false_accepts": int(np.sum(acc & (e_test > TOL))),
        "fallback_cases": int(len(rejected)), "fallback_seconds": t_fb,
        "final_max_rel_l2": float(final.max()), "final_frac_within_5pct": float(np.mean(final <= TOL + 1e-7)),
        "inference_and_gate_seconds": t_inf,
        "cases_per_s": n / (t_inf + t_fb),
        "fallback_cases_per_s": 1.0 / per_sim,
        "speedup_vs_fallback": per_sim * n / (t_inf + t_fb),
        "speedup_vs_plain": (per_plain * n / (t_inf + t_fb)) if per_plain else None,
        "gate_sweep": sweep,
        "test_rel_l2": [float(x) for x in e_test], "test_accepted": [bool(x) for x in acc],
    })
    if train_rep and "epoch_loss" in train_rep:
        rep["epoch_loss"] = train_rep["epoch_loss"]
    json.dump(rep, open(os.path.join(a.out_dir, "report.json"), "w"), indent=1)
    log(json.dumps({k_: v for k_, v in rep.items() if k_ not in ("epoch_loss", "test_rel_l2", "test_accepted",
                                                                  "gate_sweep")}, indent=1))
    for row in sweep:
        log(f"margin {row['margin']}: accepted {row['accepted_frac']:.3f}, false accepts {row['false_accepts']}, "
            f"max accepted rel-L2 {row['max_accepted_rel_l2']}")
    return rep


def pipeline(a):
    """The surrogate job (see the module docstring): phase "train", "gate",
    "test" or "all"; the test phase reads the weights and gate the train phase saved
    (--params, by default DIR/params.npz) and the training figures
    (DIR/train_report.json, else the one beside the params)."""
    import os
    os.makedirs(a.out_dir, exist_ok=True)
    log = lambda m: print(m, flush=True)
    train_rep = None
    if a.phase in ("train", "all"):
        train_rep = pipeline_train(a, log)
    if a.phase in ("gate", "all"):
        pipeline_gate(a, log, a.params or os.path.join(a.out_dir, "params.npz"))
    if a.phase in ("test", "all"):
        params = a.params or os.path.join(a.out_dir, "params.npz")
        if train_rep is None:
            for tr_path in (os.path.join(a.out_dir, "train_report.json"),
                            os.path.join(os.path.dirname(params), "train_report.json")):
                if os.path.exists(tr_path):
                    train_rep = json.load(open(tr_path))
                    break
        pipeline_test(a, log, params, train_rep)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pipeline", action="store_true", help="generate, train, gate and report")
    ap.add_argument("--phase", choices=("all", "train", "gate", "test"), default="all")
    ap.add_argument("--out-dir", default=None)
    ap.add_argument("--train-seeds", default="1000:5096")
    ap.add_argument("--test-seeds", default="9000:9512")
    ap.add_argument("--plain-sample", type=int, default=2)
    ap.add_argument("--train", default=None)
    ap.add_argument("--test", default=None)
    ap.add_argument("--out", default=None)
    ap.add_argument("--params", default=None)
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--val-frac", type=float, default=0.15)
    ap.add_argument("--k", type=int, default=3)
    ap.add_argument("--gate-margin", type=float, default=0.5,
                    help="accept a case only where its nearest validation cases are within margin * 5 %%")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--fallback", action="store_true", help="run the simulator on the rejected test cases")
    a = ap.parse_args()
    if a.pipeline:
        if not a.out_dir:
            ap.error("--pipeline needs --out-dir")
        pipeline(a)
        return
    if not (a.train and a.test and a.out):
        ap.error("--train, --test and --out are required without --pipeline")

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
        "false_accepts": int(np.sum(acc & (e_test > TOL))),
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
