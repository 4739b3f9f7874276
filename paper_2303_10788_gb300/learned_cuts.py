"""Learned cut choice: data generation, training and evaluation of the
message-passing cut scorer on the GPU.

For each circuit of the near-Clifford population (50-400 qubits, 4-40 T
gates, random interaction structure) the greedy cut search proposes
candidate cut sets; every candidate whose greedy estimate is within the
judge factor of the best one is planned, evaluated and recombined on the
GPU, and the device time of evaluation + recombination is the training
target (as its logarithm).  The scorer is trained with the library's own
forward/backward/Adam kernels.  On held-out circuits the greedy choice and
the learned choice (the library's ``use_learned`` path) are both run end to
end; their recombined marginals must agree (exact mode, cut-set invariance)
and their times are compared.

    python -m paper_2303_10788_gb300.learned_cuts --train 2000 --test 256 \\
        --weights cut_scorer.npz --report learned_cuts.json
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from workloads import Workload, config5_circuit   # noqa: E402

SEED = 230310788 + 5


def population(n, seed, marginal=10, shots=4096):
    """n seeded circuits without cut sets (the search chooses them)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        c, _, _ = config5_circuit(rng)
        marg = sorted(int(q) for q in rng.choice(c.n_qubits, size=marginal, replace=False))
        out.append(Workload(f"c5_{seed}_{i}", c, None, marg, [], shots, seed + i))
    return out


def _candidates_worker(args):
    ws, cap = args
    from paper_2303_10788_gb300 import ccs
    ctx = ccs.ccs_create(-1)
    res = []
    for w in ws:
        try:
            res.append(ccs.ccs_cut_candidates(ctx, w, cap=cap))
        except ccs.CCSError:
            res.append([])          # no cut set within the limits (counted by the callers)
    return res


def candidates(ws, cap=8, procs=None):
    """Greedy candidates [(cuts, estimate)] per circuit, on host cores (a
    spawn pool: safe before or after the GPU is in use)."""
    procs = procs or max(1, min(16, os.cpu_count() or 1))
    chunks = [ws[i::procs] for i in range(procs)]
    with mp.get_context("spawn").Pool(procs) as pool:
        parts = pool.map(_candidates_worker, [(c, cap) for c in chunks])
    out = [None] * len(ws)
    for p, part in enumerate(parts):
        for j, r in enumerate(part):
            out[p + j * procs] = r
    return out


def judged(cands, judge, max_cuts):
    """Candidates the greedy estimate allows (within `judge` of the best)."""
    if not cands:
        return []
    best = cands[0][1]
    return [(c, e) for c, e in cands if e <= judge * best and len(c) <= max_cuts]


def device_time(ctx, w, cuts, mode, reps=1):
    """Seconds of evaluation + recombination on the device for one cut set,
    after one untimed run (CUDA events on the library's stream)."""
    import torch
    from paper_2303_10788_gb300 import ccs
    ws = [Workload(w.name, w.circuit, cuts, w.marginal, w.zstrings, w.shots, w.seed)]
    plan = ccs.ccs_build_fragments(ctx, ws)
    res = ccs.ccs_eval_variants(ctx, plan, mode=mode, shots=w.shots)
    ccs.ccs_recombine(ctx, plan, res)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(reps):
        ccs.ccs_eval_variants(ctx, plan, mode=mode, shots=w.shots, res=res)
        marg, _ = ccs.ccs_recombine(ctx, plan, res)
    ev[1].record()
    torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[1]) / 1e3 / reps


def _reason(e):
    """Short label of a refused candidate (the library's error code name)."""
    msg = str(e)
    for code in ("UNSUPPORTED", "NC_TOO_WIDE", "TOO_MANY_CUTS", "INVALID_ARG", "OOM"):
        if code in msg:
            return code + (": not a star" if "star" in msg else ": hub wider than 16 bits" if "16 bits" in msg
                           else "")
    return type(e).__name__


def make_dataset(ctx, ws, cands, judge, max_cuts, log=print, dropped=None):
    """Timed samples (features, log device time) of every judged candidate.
    Candidates the library refuses are counted in ``dropped`` by reason."""
    from paper_2303_10788_gb300 import ccs
    graphs, target, groups = [], [], []
    dropped = {} if dropped is None else dropped
    t0 = time.time()
    for i, (w, cs) in enumerate(zip(ws, cands)):
        g0 = len(graphs)
        if not cs:
            dropped["no candidate"] = dropped.get("no candidate", 0) + 1
        for cuts, _ in judged(cs, judge, max_cuts):
            try:
                t = device_time(ctx, w, cuts, ccs.CCS_SAMPLED)
            except ccs.CCSError as e:
                r = _reason(e)
                dropped[r] = dropped.get(r, 0) + 1
                continue
            graphs.append(ccs.ccs_featurize(ctx, w, cuts))
            target.append(math.log(t))
        if len(graphs) > g0:
            groups.append((g0, len(graphs)))
        if (i + 1) % 100 == 0:
            log(f"  timed {i + 1}/{len(ws)} circuits, {len(graphs)} samples, {time.time() - t0:.0f} s")
    return graphs, np.asarray(target, np.float32), groups


def train(ctx, net, graphs, target, epochs, batch, lr, seed, log=print):
    from paper_2303_10788_gb300 import ccs
    rng = np.random.default_rng(seed)
    mu, sd = float(target.mean()), float(target.std() + 1e-6)
    y = (target - mu) / sd
    idx = np.arange(len(graphs))
    for ep in range(epochs):
        rng.shuffle(idx)
        losses = []
        for b0 in range(0, len(idx), batch):
            sel = idx[b0:b0 + batch]
            b = ccs.make_batch([graphs[i] for i in sel])
            losses.append(ccs.ccs_mpnn_train_step(ctx, net, b, y[sel], lr=lr))
        if ep == 0 or (ep + 1) % max(1, epochs // 10) == 0:
            log(f"  epoch {ep + 1}/{epochs}: loss {np.mean(losses):.4f}")
    return mu, sd


def predict(ctx, net, graphs, chunk=512):
    from paper_2303_10788_gb300 import ccs
    out = []
    for c0 in range(0, len(graphs), chunk):
        out.append(ccs.ccs_mpnn_forward(ctx, net, ccs.make_batch(graphs[c0:c0 + chunk])))
    return np.concatenate(out) if out else np.zeros(0, np.float32)


def e2e_time(ctx, w, learned, reps=3):
    """Median wall seconds of one circuit end to end through the C ABI: plan
    build (cut search, and with ``learned`` the scorer on the GPU picking
    among the candidates), sampled evaluation, recombination into host
    memory; after one untimed run."""
    from paper_2303_10788_gb300 import ccs
    pk = ccs.pack_problems([Workload(w.name, w.circuit, None, w.marginal, w.zstrings, w.shots, w.seed)])
    ts = []
    for i in range(reps + 1):
        t0 = time.perf_counter()
        plan = ccs.ccs_build_fragments(ctx, pk, use_learned=1 if learned else 0)
        res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=w.shots)
        ccs.ccs_recombine(ctx, plan, res)
        if i:
            ts.append(time.perf_counter() - t0)
        del res, plan
    return float(np.median(ts))


def evaluate(ctx, net, ws, cands, judge, max_cuts, check_exact=True, log=print, e2e_reps=3):
    """Greedy vs learned on held-out circuits: device time of each choice
    (evaluation + recombination, two repeats), the best measured candidate,
    exact-mode agreement of the results, and end-to-end circuits/s of the
    library's greedy and learned paths (cut search and the scorer's own cost
    included, median of ``e2e_reps`` repeats).  Candidates the library
    refuses are counted by reason."""
    from paper_2303_10788_gb300 import ccs
    rows, dropped = [], {}
    ccs.ccs_set_cut_model(ctx, net)
    for w, cs in zip(ws, cands):
        js = judged(cs, judge, max_cuts)
        if not js:
            dropped["no candidate"] = dropped.get("no candidate", 0) + 1
            continue
        feats = [ccs.ccs_featurize(ctx, w, c) for c, _ in js]
        pred = predict(ctx, net, feats)
        pick = int(np.argmin(pred))
        times = []
        for c, _ in js:
            try:
                times.append(device_time(ctx, w, c, ccs.CCS_SAMPLED, reps=2))
            except ccs.CCSError as e:
                r = _reason(e)
                dropped[r] = dropped.get(r, 0) + 1
                times.append(float("inf"))
        if not np.isfinite(times[0]) or not np.isfinite(times[pick]):
            continue
        agree = None
        if check_exact and pick != 0:
            out = []
            for c in (js[0][0], js[pick][0]):
                p = ccs.ccs_build_fragments(ctx, [Workload(w.name, w.circuit, c, w.marginal, [], w.shots, w.seed)])
                r = ccs.ccs_eval_variants(ctx, p, mode=ccs.CCS_EXACT)
                out.append(ccs.ccs_recombine(ctx, p, r)[0])
            agree = float(np.abs(out[0] - out[1]).max())
        row = {"greedy": times[0], "learned": times[pick], "best": float(min(times)),
               "changed": pick != 0, "n_cands": len(js), "max_abs_diff": agree}
        if e2e_reps:
            try:
                row["e2e_greedy"] = e2e_time(ctx, w, False, e2e_reps)
                row["e2e_learned"] = e2e_time(ctx, w, True, e2e_reps)
            except ccs.CCSError as e:       # the library's own pick refused (counted, left out)
                row.pop("e2e_greedy", None)
                r = "end to end: " + _reason(e)
                dropped[r] = dropped.get(r, 0) + 1
        rows.append(row)
    ccs.ccs_set_cut_model(ctx, None)
    g = sum(r["greedy"] for r in rows)
    l = sum(r["learned"] for r in rows)
    b = sum(r["best"] for r in rows)
    both = [r for r in rows if "e2e_learned" in r]
    eg = sum(r["e2e_greedy"] for r in both)
    el = sum(r["e2e_learned"] for r in both)
    diffs = [r["max_abs_diff"] for r in rows if r["max_abs_diff"] is not None]
    return {"circuits": len(rows), "greedy_circuits_per_s": len(rows) / g if g else 0.0,
            "learned_circuits_per_s": len(rows) / l if l else 0.0,
            "best_candidate_circuits_per_s": len(rows) / b if b else 0.0,
            "speedup_learned_over_greedy": g / l if l else 0.0,
            "e2e_circuits": len(both),
            "e2e_greedy_circuits_per_s": len(both) / eg if eg else 0.0,
            "e2e_learned_circuits_per_s": len(both) / el if el else 0.0,
            "e2e_speedup_learned_over_greedy": eg / el if el else 0.0,
            "picks_changed": sum(r["changed"] for r in rows),
            "dropped_candidates": dropped,
            "max_abs_diff_exact": max(diffs) if diffs else 0.0,
            "rows": rows}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=256)
    ap.add_argument("--cands", type=int, default=8)
    ap.add_argument("--judge", type=float, default=16.0)
    ap.add_argument("--max-cuts", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=SEED)
    ap.add_argument("--weights", default=None, help="write the trained parameters (npz)")
    ap.add_argument("--load", default=None, help="evaluate these trained parameters (npz) instead of training")
    ap.add_argument("--report", default=None, help="write the evaluation report (json)")
    a = ap.parse_args(argv)
    t0 = time.time()
    ws_tr = population(a.train, a.seed) if not a.load else []
    ws_te = population(a.test, a.seed + 1_000_003)
    c_tr = candidates(ws_tr, a.cands) if ws_tr else []
    c_te = candidates(ws_te, a.cands)
    print(f"candidates: {time.time() - t0:.0f} s", flush=True)
    from paper_2303_10788_gb300 import ccs
    ctx = ccs.ccs_create(0)
    dropped = {}
    if a.load:
        net = ccs.load_cut_scorer(ctx, a.load)
        graphs, mu, sd = [], float("nan"), float("nan")
    else:
        graphs, target, _ = make_dataset(ctx, ws_tr, c_tr, a.judge, a.max_cuts, dropped=dropped)
        print(f"dataset: {len(graphs)} samples, {time.time() - t0:.0f} s; dropped {dropped}", flush=True)
        net = ccs.ccs_mpnn_create(ctx, seed=a.seed)
        mu, sd = train(ctx, net, graphs, target, a.epochs, a.batch, a.lr, a.seed)
    rep = evaluate(ctx, net, ws_te, c_te, a.judge, a.max_cuts)
    rep.update({"train_circuits": 0 if a.load else a.train, "loaded": a.load, "train_samples": len(graphs),
                "train_dropped_candidates": dropped,
                "target_mean": mu, "target_std": sd, "seconds": time.time() - t0})
    print(json.dumps({k: v for k, v in rep.items() if k != "rows"}), flush=True)
    if a.weights:
        np.savez(a.weights, params=ccs.ccs_mpnn_params(ctx, net), target_mean=mu, target_std=sd)
    if a.report:
        with open(a.report, "w") as f:
            json.dump(rep, f, indent=1)
    return rep


if __name__ == "__main__":
    main()
