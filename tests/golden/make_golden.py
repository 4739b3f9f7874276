"""Writes the stored oracle results under tests/golden/ (calls only ``oracle/``).

Sampled-mode recombined marginals of the largest workloads, with the
canonical outcome space (rank, offset, basis; Sec. V-B's per-variant output
distribution is uniform on it) of every Clifford variant, for the seed the
benchmark uses.  The GPU tests compare the library's default evaluation path
with these values; nothing here reads the library.

    python tests/golden/make_golden.py config3 [--procs 8]
    python tests/golden/make_golden.py config4 [--procs 8] [--circuits 0,1,...]
    python tests/golden/make_golden.py exact [--procs 8]
    python tests/golden/make_golden.py ml [--procs 8]

``exact`` (after the two above) writes the exact-mode marginals (strong
simulation, Sec. V-C: each Clifford variant's distribution is 2^-rank on its
outcome space) of the same circuits from the stored oracle outcome spaces,
so no tableau is simulated again.

``ml`` (after ``config4``) writes the sampled-mode marginals of the stored
config-4 circuits with every Clifford fragment's model corrected by maximum
likelihood (Sec. V-C; ``oracle.mlcorrect``) before the contraction: the
shot counts are drawn again from the stored outcome spaces with the same
Philox stream, folded, corrected and contracted.

config3 (500-qubit body, 20736 variants, 2^14 shots, 4^8 cut terms) takes
about 5 CPU-hours; it is spread over ``--procs`` spawned processes.  Each
variant is the circuit (preparations, body gates, basis changes); the
preparations and body are run once per preparation combination and the
basis changes applied to copies of that tableau, which is the same gate
sequence.  The body tensor is folded column block by column block: the
columns whose output Paulis P_out share one basis combination beta(P_out)
need only the variants measured in that combination (the fold's definition),
so each block is one task.
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

SEED = (0x9E3779B9, 0x7F4A7C15)     # the benchmark's (seed_lo, seed_hi) at rank 0


def _space_row(off, B, rank, width=26):
    row = np.zeros(width, np.uint32)
    row[0], row[1] = rank, off
    row[2:2 + len(B)] = B
    return row


# --- config 3 ---------------------------------------------------------------

def _c3_setup(name="config3"):
    import workloads
    from oracle.cutting import fragment_circuit
    w = getattr(workloads, name)()
    frags, cuts = fragment_circuit(w.circuit, w.cuts, w.marginal)
    body = max(range(len(frags)), key=lambda i: frags[i].n)
    return w, frags, cuts, body


def _c3_prefix(args):
    """Tableau after the preparations of combination ``s_idx`` and the body."""
    s_idx, tmp, name = args
    from oracle import tableau as tb
    from oracle.cutting import PREP_GATES
    w, frags, _, body = _c3_setup(name)
    f = frags[body]
    g = []
    for j, (_, wire) in enumerate(f.qin):
        g += [(op, wire, -1) for op in PREP_GATES[(s_idx >> (2 * j)) & 3]]
    tab = tb.Tableau(f.n).run(g + list(f.gates))
    np.savez(os.path.join(tmp, f"pre{s_idx}.npz"), x=tab.x, z=tab.z, r=tab.r)
    return s_idx


def _c3_block(args):
    """One basis combination: its 4^qin variants' outcome spaces and shots,
    and the body tensor's columns measured in it."""
    b_idx, tmp, name = args
    from oracle import tableau as tb
    from oracle.cutting import BASIS_GATES, BETA, fold_columns, pauli_digits
    from oracle.pipeline import sample_counts
    w, frags, _, body = _c3_setup(name)
    f = frags[body]
    nin = 4 ** len(f.qin)
    beta = f.variant_digits(b_idx * nin)[1]
    dists, spaces = {}, {}
    for s_idx in range(nin):
        v = s_idx + nin * b_idx
        d = np.load(os.path.join(tmp, f"pre{s_idx}.npz"))
        tab = tb.Tableau.__new__(tb.Tableau)
        tab.n, tab.x, tab.z, tab.r = f.n, d["x"].copy(), d["z"].copy(), d["r"].copy()
        for (_, wire), bj in zip(f.qout, beta):
            for op in BASIS_GATES[bj]:
                tab.apply(op, wire)
        off, B, rho = tb.outcome_space(tab, f.A)
        counts = sample_counts(off, B, len(f.A), w.shots, v, body, 0, SEED[0], SEED[1])
        dists[v] = counts / float(w.shots)
        spaces[v] = _space_row(off, B, rho)
    Ps = [P for P in range(4 ** len(f.slots))
          if [BETA[p] for p in pauli_digits(f, P)[1]] == beta]
    cols = fold_columns(f, Ps, lambda v: dists[v])
    return b_idx, Ps, cols, spaces


def make_config3(procs, name="config3", out=None):
    """Star with one Clifford hub and statevector leaves (config 3's shape;
    ``name`` = another such workload for a check of this route)."""
    from oracle import statevector as sv
    from oracle.cutting import fold, recombine
    w, frags, cuts, body = _c3_setup(name)
    f = frags[body]
    nin, nout = 4 ** len(f.qin), 3 ** len(f.qout)
    t0 = time.time()
    tensors = []
    for fi, fr in enumerate(frags):
        if fi == body:
            tensors.append(None)
            continue
        assert not fr.clifford
        dists = [sv.marginal(sv.run(fr.n, fr.variant_gates(v)), fr.n, fr.A) for v in range(fr.n_variants)]
        tensors.append(fold(fr, dists))
    spaces = np.zeros((f.n_variants, 26), np.uint32)
    Tb = np.zeros((1 << len(f.marg), 4 ** len(f.slots)))
    with tempfile.TemporaryDirectory() as tmp, mp.get_context("spawn").Pool(procs) as pool:
        for _ in pool.imap_unordered(_c3_prefix, [(s, tmp, name) for s in range(nin)]):
            pass
        print(f"prefix tableaus: {time.time() - t0:.0f} s", flush=True)
        for done, (b_idx, Ps, cols, sp) in enumerate(
                pool.imap_unordered(_c3_block, [(b, tmp, name) for b in range(nout)])):
            Tb[:, Ps] = cols
            for v, row in sp.items():
                spaces[v] = row
            print(f"block {b_idx} ({done + 1}/{nout}): {time.time() - t0:.0f} s", flush=True)
    tensors[body] = Tb
    marg = recombine(frags, tensors, len(cuts), len(w.marginal))
    print(f"recombined: {time.time() - t0:.0f} s; sum {marg.sum():.6f}", flush=True)
    if out is None:
        return marg, spaces
    np.savez_compressed(out, marginal=marg, spaces=spaces, body=np.int64(body),
                        seed=np.array(SEED, np.uint64), shots=np.int64(w.shots))
    print("wrote", out)


# --- config 4 ---------------------------------------------------------------

def _c4_one(ci):
    from workloads import config4
    from oracle.pipeline import evaluate_workload
    w = config4(256)[ci]
    r = evaluate_workload(w, mode="sampled", seed_lo=SEED[0], seed_hi=SEED[1], circuit_id=ci,
                          keep_tableaus=False)
    sp = []
    for fi, fr in enumerate(r.fragments):
        if fr.clifford:
            for v, vr in enumerate(r.variants[fi]):
                sp.append(np.concatenate([[fi, v], _space_row(vr.off, vr.basis, len(vr.basis))]))
    return ci, r.marginal, np.array(sp, np.uint32)


def make_config4(procs, circuits):
    t0 = time.time()
    margs, spaces = {}, {}
    with mp.get_context("spawn").Pool(procs) as pool:
        for ci, m, sp in pool.imap_unordered(_c4_one, circuits):
            margs[ci], spaces[ci] = m, sp
            print(f"circuit {ci}: {time.time() - t0:.0f} s", flush=True)
    out = os.path.join(HERE, "config4_sampled.npz")
    np.savez_compressed(out, circuits=np.array(circuits, np.int64),
                        marginals=np.stack([margs[c] for c in circuits]),
                        **{f"spaces_{c}": spaces[c] for c in circuits},
                        seed=np.array(SEED, np.uint64))
    print("wrote", out)


# --- exact mode from the stored outcome spaces -----------------------------------

def _exact_dist(row, nbits):
    from oracle import tableau as tb
    rank, off = int(row[0]), int(row[1])
    return tb.exact_distribution(off, [int(b) for b in row[2:2 + rank]], nbits)


def _c3_exact_block(b_idx):
    from oracle.cutting import BETA, fold_columns, pauli_digits
    w, frags, _, body = _c3_setup()
    f = frags[body]
    nin = 4 ** len(f.qin)
    beta = f.variant_digits(b_idx * nin)[1]
    sp = np.load(os.path.join(HERE, "config3_sampled.npz"))["spaces"]
    dists = {v: _exact_dist(sp[v], len(f.A)) for v in range(b_idx * nin, (b_idx + 1) * nin)}
    Ps = [P for P in range(4 ** len(f.slots))
          if [BETA[p] for p in pauli_digits(f, P)[1]] == beta]
    return Ps, fold_columns(f, Ps, lambda v: dists[v])


def _c4_exact_one(ci):
    from workloads import config4
    from oracle import statevector as sv
    from oracle.cutting import fragment_circuit, fold, recombine
    w = config4(256)[ci]
    frags, cuts = fragment_circuit(w.circuit, w.cuts, w.marginal)
    rows = np.load(os.path.join(HERE, "config4_sampled.npz"))[f"spaces_{ci}"]
    by = {(int(r[0]), int(r[1])): r[2:] for r in rows}
    tensors = []
    for fi, fr in enumerate(frags):
        if fr.clifford:
            dists = [_exact_dist(by[(fi, v)], len(fr.A)) for v in range(fr.n_variants)]
        else:
            dists = [sv.marginal(sv.run(fr.n, fr.variant_gates(v)), fr.n, fr.A) for v in range(fr.n_variants)]
        tensors.append(fold(fr, dists))
    return ci, recombine(frags, tensors, len(cuts), len(w.marginal))


def _c4_ml_one(ci):
    from workloads import config4
    from oracle import statevector as sv
    from oracle.cutting import fragment_circuit, fold, recombine
    from oracle.mlcorrect import ml_correct
    from oracle.pipeline import sample_counts
    w = config4(256)[ci]
    frags, cuts = fragment_circuit(w.circuit, w.cuts, w.marginal)
    rows = np.load(os.path.join(HERE, "config4_sampled.npz"))[f"spaces_{ci}"]
    by = {(int(r[0]), int(r[1])): r[2:] for r in rows}
    tensors = []
    for fi, fr in enumerate(frags):
        if fr.clifford:
            dists = []
            for v in range(fr.n_variants):
                row = by[(fi, v)]
                rank, off = int(row[0]), int(row[1])
                c = sample_counts(off, [int(b) for b in row[2:2 + rank]], len(fr.A), w.shots, v, fi, ci,
                                  SEED[0], SEED[1])
                dists.append(c / float(w.shots))
            tensors.append(ml_correct(fr, fold(fr, dists))[0])
        else:
            dists = [sv.marginal(sv.run(fr.n, fr.variant_gates(v)), fr.n, fr.A) for v in range(fr.n_variants)]
            tensors.append(fold(fr, dists))
    return ci, recombine(frags, tensors, len(cuts), len(w.marginal))


def make_ml(procs):
    t0 = time.time()
    g4 = np.load(os.path.join(HERE, "config4_sampled.npz"))
    circuits = [int(c) for c in g4["circuits"]]
    m = {}
    with mp.get_context("spawn").Pool(procs) as pool:
        for ci, mc in pool.imap_unordered(_c4_ml_one, circuits):
            m[ci] = mc
            print(f"circuit {ci}: {time.time() - t0:.0f} s", flush=True)
    out = os.path.join(HERE, "ml_marginals.npz")
    np.savez_compressed(out, config4_circuits=np.array(circuits, np.int64),
                        config4=np.stack([m[c] for c in circuits]), seed=np.array(SEED, np.uint64))
    print("wrote", out)


def make_exact(procs):
    from oracle import statevector as sv
    from oracle.cutting import fold, recombine
    t0 = time.time()
    w, frags, cuts, body = _c3_setup()
    f = frags[body]
    tensors = [None if fi == body else
               fold(fr, [sv.marginal(sv.run(fr.n, fr.variant_gates(v)), fr.n, fr.A) for v in range(fr.n_variants)])
               for fi, fr in enumerate(frags)]
    Tb = np.zeros((1 << len(f.marg), 4 ** len(f.slots)))
    g4 = np.load(os.path.join(HERE, "config4_sampled.npz"))
    circuits = [int(c) for c in g4["circuits"]]
    m4 = {}
    with mp.get_context("spawn").Pool(procs) as pool:
        r4 = pool.map_async(_c4_exact_one, circuits)
        for Ps, cols in pool.imap_unordered(_c3_exact_block, range(3 ** len(f.qout))):
            Tb[:, Ps] = cols
        print(f"config3 blocks: {time.time() - t0:.0f} s", flush=True)
        for ci, m in r4.get():
            m4[ci] = m
    tensors[body] = Tb
    m3 = recombine(frags, tensors, len(cuts), len(w.marginal))
    print(f"config3 recombined: {time.time() - t0:.0f} s; sum {m3.sum():.9f}", flush=True)
    out = os.path.join(HERE, "exact_marginals.npz")
    np.savez_compressed(out, config3=m3, config4_circuits=np.array(circuits, np.int64),
                        config4=np.stack([m4[c] for c in circuits]))
    print("wrote", out)


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["config3", "config4", "exact", "ml"])
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--circuits", default="0,1,2,3,4,5,6,7")
    a = ap.parse_args()
    if a.which == "config3":
        make_config3(a.procs, out=os.path.join(HERE, "config3_sampled.npz"))
    elif a.which == "config4":
        make_config4(a.procs, [int(c) for c in a.circuits.split(",")])
    elif a.which == "ml":
        make_ml(a.procs)
    else:
        make_exact(a.procs)
