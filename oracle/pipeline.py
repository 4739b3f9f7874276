"""ORACLE (test infrastructure): the whole path on one circuit, plainly.

Follows the paper's flow (Sec. V): cut the circuit (Sec. V-A), evaluate every
variant of every fragment -- Clifford fragments by a stabilizer tableau,
non-Clifford ones by an exact statevector (Sec. V-B) -- and rebuild the
distribution of the uncut circuit by contracting the fragment tensors
(Sec. V-C).  The maximum-likelihood correction of the fragment models is a
separate step (``oracle.mlcorrect.ml_correct`` on ``OracleResult.tensors``).

Modes: ``"exact"`` uses the closed-form 2^-rank distribution of each Clifford
variant (strong simulation, Sec. V-C last paragraph); ``"sampled"`` draws
``shots`` Philox shots per Clifford variant from its affine outcome space.
Non-Clifford variants are always exact.

Z-string expectations <Z_S> are contracted from per-fragment one-dimensional
tensors: for each variant and each subset u of quantum outputs, the
expectation of Z on (S's wires in the fragment) + u.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import tableau as tb
from . import statevector as sv
from .cutting import fragment_circuit, fold, fold_scalar, recombine, recombine_scalar
from .philox import shot_coeffs


@dataclass
class VariantResult:
    dist: np.ndarray                 # float64 over 2^|A|
    tableau: np.ndarray | None = None   # uint8 [2n, 2n+1] (Clifford only)
    off: int | None = None
    basis: list | None = None
    counts: np.ndarray | None = None    # int64 over 2^|A| (sampled mode)
    zvals: np.ndarray | None = None     # [n_z, 2^q_out]


@dataclass
class OracleResult:
    fragments: list
    cuts: list
    variants: list                   # [fragment][variant] -> VariantResult
    tensors: list
    marginal: np.ndarray
    zexp: np.ndarray
    meta: dict = field(default_factory=dict)


def sample_counts(off, B, nbits, shots, variant, fragment, circuit, seed_lo, seed_hi):
    """Counts of y = off ^ XOR_{j: c_j = 1} B_j with c = the shot's rho
    coefficient bits from the Philox stream (``shot_coeffs``, rho <= 24)."""
    assert len(B) <= 24
    bits = shot_coeffs(shots, len(B), variant, fragment, circuit, seed_lo, seed_hi)
    y = np.full(shots, off, np.int64)
    for j, b in enumerate(B):
        sel = ((bits >> np.uint64(j)) & np.uint64(1)).astype(bool)
        y[sel] ^= b
    return np.bincount(y, minlength=1 << nbits).astype(np.int64)


def evaluate(circuit, cuts, marginal, zstrings=(), mode="sampled", shots=1024,
             seed_lo=0x1234, seed_hi=0x5678, circuit_id=0, variants_only=None,
             keep_tableaus=True):
    frags, cuts_c = fragment_circuit(circuit, cuts, marginal)
    k = len(cuts_c)
    # which fragment holds each qubit's final segment
    n_seg = {q: 1 + sum(1 for (qq, _) in cuts_c if qq == q) for q in range(circuit.n_qubits)}
    out_wire = {}
    for fi, f in enumerate(frags):
        for li, (q, kk) in enumerate(f.wires):
            if kk == n_seg[q] - 1:
                out_wire[q] = (fi, li)
    results = []
    for fi, f in enumerate(frags):
        A = f.A
        rs = []
        vlist = range(f.n_variants) if variants_only is None else variants_only.get(fi, [])
        for v in vlist:
            gates = f.variant_gates(v)
            zv = np.zeros((len(zstrings), 1 << len(f.qout)))
            if f.clifford:
                tab = tb.Tableau(f.n).run(gates)
                off, B, rho = tb.outcome_space(tab, A)
                if mode == "exact":
                    dist = tb.exact_distribution(off, B, len(A))
                    counts = None
                else:
                    counts = sample_counts(off, B, len(A), shots, v, fi, circuit_id, seed_lo, seed_hi)
                    dist = counts / float(shots)
                supp = tb.support(tab) if len(zstrings) else None
                for si, zs in enumerate(zstrings):
                    base = [out_wire[q][1] for q in zs if out_wire[q][0] == fi]
                    for u in range(1 << len(f.qout)):
                        ws = base + [w for j, (_, w) in enumerate(f.qout) if (u >> j) & 1]
                        zv[si, u] = tb.z_expectation(tab, ws, supp)
                rs.append(VariantResult(dist, tb.tableau_bits(tab) if keep_tableaus else None,
                                        off, B, counts, zv))
            else:
                psi = sv.run(f.n, gates)
                dist = sv.marginal(psi, f.n, A)
                for si, zs in enumerate(zstrings):
                    base = [out_wire[q][1] for q in zs if out_wire[q][0] == fi]
                    for u in range(1 << len(f.qout)):
                        ws = base + [w for j, (_, w) in enumerate(f.qout) if (u >> j) & 1]
                        zv[si, u] = sv.z_expectation(psi, f.n, ws)
                rs.append(VariantResult(dist, zvals=zv))
        results.append(rs)
    if variants_only is not None:
        return OracleResult(frags, cuts_c, results, [], np.zeros(0), np.zeros(0))
    tensors = [fold(f, [r.dist for r in rs]) for f, rs in zip(frags, results)]
    marg = recombine(frags, tensors, k, len(marginal))
    zexp = np.zeros(len(zstrings))
    for si in range(len(zstrings)):
        ts = [fold_scalar(f, [r.zvals[si] for r in rs]) for f, rs in zip(frags, results)]
        zexp[si] = recombine_scalar(frags, ts, k)
    return OracleResult(frags, cuts_c, results, tensors, marg, zexp,
                        {"k": k, "mode": mode, "shots": shots})


def evaluate_workload(w, mode="sampled", seed_lo=0x1234, seed_hi=0x5678, circuit_id=0, **kw):
    return evaluate(w.circuit, w.cuts, w.marginal, w.zstrings, mode, w.shots,
                    seed_lo, seed_hi, circuit_id, **kw)


def brute_force(circuit, marginal, zstrings=()):
    """Uncut dense statevector: marginal and Z-string expectations (n <= ~20)."""
    psi = sv.run(circuit.n_qubits, circuit.gates)
    return (sv.marginal(psi, circuit.n_qubits, list(marginal)),
            np.array([sv.z_expectation(psi, circuit.n_qubits, list(z)) for z in zstrings]))


def uncut_clifford(circuit, marginal, zstrings=()):
    """Closed-form marginal of one uncut tableau (the circuit must be Clifford)."""
    tab = tb.Tableau(circuit.n_qubits).run(circuit.gates)
    off, B, _ = tb.outcome_space(tab, list(marginal))
    return (tb.exact_distribution(off, B, len(marginal)),
            np.array([tb.z_expectation(tab, list(z)) for z in zstrings]))
