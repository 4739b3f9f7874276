"""ORACLE (test infrastructure): wire cuts, fragments, variants, fold, recombination.

Circuit cutting (Sec. III-B): each cut splits a wire; the upstream fragment
gets a *quantum output* there, measured in several bases, and the downstream
fragment a *quantum input*, prepared in several states (Sec. V-B's four I/O
kinds).  One *variant* fixes a preparation at every quantum input and a basis
at every quantum output; a fragment has 4^{q_in} 3^{q_out} of them.  The
fragment results are stitched together by a contraction with one tensor per
fragment and one edge per cut, costing ~4^k (Sec. III-B, Sec. V-C).

The decomposition is written in the Pauli basis (Sec. III-B): on a cut wire
  rho = 1/2 sum_{P in {I,X,Y,Z}} Tr(P rho) P.
Upstream, Tr(P rho) is read by measuring in basis beta(P) (Z for I and Z) and
weighting outcome b by lambda_P(b) = 1 for I, (-1)^b otherwise.  Downstream,
P is expanded in prepared states: I = |0><0| + |1><1|,  Z = |0><0| - |1><1|,
X = 2|+><+| - |0><0| - |1><1|,  Y = 2|+i><+i| - |0><0| - |1><1|.
Then p(o) = 2^-k sum_{P in 4^k} prod_f T_f(o_f, P|f) with
  T_f(o, P) = sum_s prod_i mu(P_in_i, s_i) sum_b prod_j lambda(P_out_j, b_j)
              p_{(s, beta(P_out))}(o, b).

Conventions shared with the C ABI (they are part of the interface):
  * a cut (q, g) splits qubit q's wire just before gate index g; cuts are
    ordered by (g, q);
  * wires (segments) of a fragment are ordered by (qubit, segment index);
    fragments by their first wire;
  * preparations 0..3 = |0>, |1>, |+>, |+i>; bases 0..2 = X, Y, Z; Paulis
    0..3 = I, X, Y, Z;
  * variant id = mixed radix, quantum inputs first (radix 4, first input
    least significant), then quantum outputs (radix 3), both in cut order;
  * measured list A_f = marginal wires of f (marginal order) then quantum
    output wires (cut order); y bit j = A_f[j];
  * T_f's Pauli index = sum_j p_j 4^j over the cuts incident to f in cut order.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from workloads import H, S, SDG, X, Y, Z, CX, CZ, T, TDG, ZPOW, NQ, gate_param

PREP_GATES = {0: [], 1: [X], 2: [H], 3: [H, S]}          # |0>,|1>,|+>,|+i>
BASIS_GATES = {0: [H], 1: [SDG, H], 2: []}               # X, Y, Z
# mu[P][s]: P expanded in prepared states s (rows I, X, Y, Z).
MU = np.array([[1, 1, 0, 0],
               [-1, -1, 2, 0],
               [-1, -1, 0, 2],
               [1, -1, 0, 0]], np.float64)
BETA = [2, 0, 1, 2]                                       # basis of P: I->Z, X, Y, Z


@dataclass
class Fragment:
    wires: list                  # (qubit, segment)
    gates: list                  # (op, a, b) or (ZPOW, a, -1, exponent) on local wires
    qin: list                    # (cut id, local wire), cut order
    qout: list                   # (cut id, local wire), cut order
    marg: list                   # (marginal position, local wire), marginal order
    clifford: bool = True
    slots: list = field(default_factory=list)   # incident cut ids, ascending

    @property
    def n(self):
        return len(self.wires)

    @property
    def A(self):
        return [w for _, w in self.marg] + [w for _, w in self.qout]

    @property
    def n_variants(self):
        return 4 ** len(self.qin) * 3 ** len(self.qout)

    def variant_digits(self, v):
        s, b = [], []
        for _ in self.qin:
            s.append(v % 4); v //= 4
        for _ in self.qout:
            b.append(v % 3); v //= 3
        return s, b

    def variant_gates(self, v):
        s, beta = self.variant_digits(v)
        g = []
        for (_, w), si in zip(self.qin, s):
            g += [(op, w, -1) for op in PREP_GATES[si]]
        g += list(self.gates)
        for (_, w), bi in zip(self.qout, beta):
            g += [(op, w, -1) for op in BASIS_GATES[bi]]
        return g


def is_clifford_gate(g):
    """T and T^dagger are not Clifford; Z^a is Clifford exactly when 2a is an
    integer (then Z^a = S^{2a}, Sec. II-C); every other opcode is."""
    if g[0] in (T, TDG):
        return False
    if g[0] == ZPOW:
        k = 2.0 * gate_param(g)
        return k == np.floor(k)
    return True


def canonical_cuts(cuts):
    cs = sorted({(int(q), int(g)) for q, g in cuts}, key=lambda c: (c[1], c[0]))
    return cs


def fragment_circuit(circuit, cuts, marginal):
    """Split ``circuit`` at ``cuts``; returns (fragments, canonical cuts)."""
    n = circuit.n_qubits
    gates = circuit.gates
    cuts = canonical_cuts(cuts)
    pos = {q: sorted(g for (qq, g) in cuts if qq == q) for q in range(n)}

    def seg(q, g):
        return sum(1 for p in pos[q] if p <= g)

    segs = [(q, k) for q in range(n) for k in range(len(pos[q]) + 1)]
    parent = {s: s for s in segs}

    def find(s):
        while parent[s] != s:
            parent[s] = parent[parent[s]]
            s = parent[s]
        return s

    for gi, g in enumerate(gates):
        op, a, b = g[:3]
        if NQ[op] == 2:
            ra, rb = find((a, seg(a, gi))), find((b, seg(b, gi)))
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
    groups = {}
    for s in segs:
        groups.setdefault(find(s), []).append(s)
    order = sorted(groups, key=lambda r: min(groups[r]))
    frags = []
    where = {}
    for fi, root in enumerate(order):
        wires = sorted(groups[root])
        for li, s in enumerate(wires):
            where[s] = (fi, li)
        frags.append(Fragment(wires, [], [], [], []))
    for gi, g in enumerate(gates):
        op, a, b = g[:3]
        fa, la = where[(a, seg(a, gi))]
        if NQ[op] == 2:
            fb, lb = where[(b, seg(b, gi))]
            assert fa == fb
            frags[fa].gates.append((op, la, lb))
        else:
            frags[fa].gates.append((op, la, -1) + tuple(g[3:]))
            if not is_clifford_gate(g):
                frags[fa].clifford = False
    for ci, (q, g) in enumerate(cuts):
        k = pos[q].index(g) + 1
        fu, lu = where[(q, k - 1)]
        fd, ld = where[(q, k)]
        if fu == fd:
            raise ValueError("a cut whose two ends lie in one fragment is not supported")
        frags[fu].qout.append((ci, lu))
        frags[fd].qin.append((ci, ld))
        frags[fu].slots.append(ci)
        frags[fd].slots.append(ci)
    for mi, q in enumerate(marginal):
        f, l = where[(q, len(pos[q]))]
        frags[f].marg.append((mi, l))
    for f in frags:
        f.slots.sort()
    return frags, cuts


def fold(frag, dists):
    """T_f[o, P] from per-variant distributions ``dists[v][y]`` (float64).

    y = o | b << m with m marginal bits and b the quantum-output bits.
    """
    dists = np.asarray(dists, np.float64)
    return fold_columns(frag, range(4 ** len(frag.slots)), lambda v: dists[v])


def pauli_digits(frag, P):
    """Split a fragment Pauli index into (P_in per quantum input, P_out per
    quantum output), both in cut order."""
    pin = [0] * len(frag.qin)
    pout = [0] * len(frag.qout)
    role = {c: ("in", j) for j, (c, _) in enumerate(frag.qin)}
    role.update({c: ("out", j) for j, (c, _) in enumerate(frag.qout)})
    for j, c in enumerate(frag.slots):
        pj = (P >> (2 * j)) & 3
        kind, idx = role[c]
        if kind == "in":
            pin[idx] = pj
        else:
            pout[idx] = pj
    return pin, pout


def fold_columns(frag, Ps, dist_of):
    """Columns T_f[:, P] for the Pauli indices ``Ps`` (in that order), each by
    the definition above: the variants measured in basis beta(P_out),
    weighted by prod mu(P_in, s) and, per outcome b of the quantum outputs,
    prod lambda(P_out, b).  ``dist_of(v)`` returns variant v's distribution;
    only the variants a column needs are asked for."""
    m = len(frag.marg)
    qo = len(frag.qout)
    Ps = list(Ps)
    T_ = np.zeros((1 << m, len(Ps)))
    o_idx = np.arange(1 << m)
    for col, P in enumerate(Ps):
        pin, pout = pauli_digits(frag, P)
        beta = [BETA[p] for p in pout]
        acc = np.zeros(1 << m)
        for v in range(frag.n_variants):
            s, bv = frag.variant_digits(v)
            if bv != beta:
                continue
            coef = 1.0
            for pi_, si in zip(pin, s):
                coef *= MU[pi_, si]
            if coef == 0.0:
                continue
            dv = dist_of(v)
            for b in range(1 << qo):
                lam = 1.0
                for j, pj in enumerate(pout):
                    if pj != 0 and (b >> j) & 1:
                        lam = -lam
                acc += coef * lam * dv[o_idx | (b << m)]
        T_[:, col] = acc
    return T_


def fold_scalar(frag, values):
    """Fold for one-dimensional fragment outputs: ``values[v][u]`` is the
    expectation of a sign (-1)^{...} times (-1)^{sum_{j in u} b_j} for the
    quantum-output subset u (bitmask); returns T[P]."""
    qi, qo = len(frag.qin), len(frag.qout)
    role = {}
    for j, (c, _) in enumerate(frag.qin):
        role[c] = ("in", j)
    for j, (c, _) in enumerate(frag.qout):
        role[c] = ("out", j)
    nslot = len(frag.slots)
    out = np.zeros(4 ** nslot)
    for P in range(4 ** nslot):
        pin = [0] * qi
        pout = [0] * qo
        for j, c in enumerate(frag.slots):
            pj = (P >> (2 * j)) & 3
            kind, idx = role[c]
            if kind == "in":
                pin[idx] = pj
            else:
                pout[idx] = pj
        beta = [BETA[p] for p in pout]
        u = sum(1 << j for j, p in enumerate(pout) if p != 0)
        acc = 0.0
        for v in range(frag.n_variants):
            s, bv = frag.variant_digits(v)
            if bv != beta:
                continue
            coef = 1.0
            for pi_, si in zip(pin, s):
                coef *= MU[pi_, si]
            acc += coef * values[v][u]
        out[P] = acc
    return out


def recombine(frags, tensors, k, n_marg):
    """p(o) = 2^-k sum_P prod_f T_f(o_f, P|f), summed naively over P in chunks."""
    p = np.zeros(1 << n_marg)
    o = np.arange(1 << n_marg)
    chunk = 256
    for P0 in range(0, 4 ** k, chunk):
        Ps = np.arange(P0, min(4 ** k, P0 + chunk))
        prod = np.ones((1 << n_marg, len(Ps)))
        for f, Tf in zip(frags, tensors):
            of = np.zeros(1 << n_marg, np.int64)
            for j, (mi, _) in enumerate(f.marg):
                of |= ((o >> mi) & 1) << j
            pf = np.zeros(len(Ps), np.int64)
            for j, c in enumerate(f.slots):
                pf |= ((Ps >> (2 * c)) & 3) << (2 * j)
            prod *= Tf[of[:, None], pf[None, :]]
        p += prod.sum(axis=1)
    return p / 2.0 ** k


def recombine_scalar(frags, tensors, k):
    tot = 0.0
    Ps = np.arange(4 ** k)
    prod = np.ones(len(Ps))
    for f, Tf in zip(frags, tensors):
        pf = np.zeros(len(Ps), np.int64)
        for j, c in enumerate(f.slots):
            pf |= ((Ps >> (2 * c)) & 3) << (2 * j)
        prod = prod * Tf[pf]
    tot = prod.sum()
    return tot / 2.0 ** k
