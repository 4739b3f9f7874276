"""Seeded near-Clifford circuit generators shaped like the paper's workloads.

Circuits follow the paper's near-Clifford setting (Sec. III-A, Sec. IV): a
Clifford body with a few T = Z^{1/4} gates (Sec. II-C), or other Z^a
rotations (Sec. VIII).  Gates are stored as ``(op, q0, q1)`` tuples
(``q1 = -1`` for one-qubit gates) using the opcodes below, which match
``ccs_gate.op`` in ``include/ccs.h``; a Z^a gate carries its exponent as a
fourth entry, ``(ZPOW, q, -1, a)``.

The partition is fixed first (a "star"): each non-Clifford region is a set of
full qubits plus a time window of one boundary qubit, i.e. two wire cuts per
region, the boundary qubit being cut out of the middle of the Clifford body
(Sec. III-B, Fig. 2 caption).  Brickwork pairs that straddle a fragment
boundary are never formed: at each layer brickwork pairs are drawn within
each fragment's qubits, so the intended cut set isolates every T gate.

Uniform random two-qubit Cliffords are drawn with the double-coset form
C2 = U (C1 x C1) g_c (C1 x C1) over the four local-equivalence classes
(identity, CNOT, double-CNOT, SWAP) of sizes 576, 5184, 5184, 576; with both
local factors uniform, the product is uniform over each double coset.  Only
gate words are produced here; no Pauli or tableau arithmetic is done.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Opcodes (ccs_gate.op).
H, S, SDG, X, Y, Z, CX, CZ, T, TDG, ZPOW = range(11)
GATE_NAMES = ["H", "S", "SDG", "X", "Y", "Z", "CX", "CZ", "T", "TDG", "ZPOW"]
NQ = [1, 1, 1, 1, 1, 1, 2, 2, 1, 1, 1]


def gate_param(g):
    """The exponent of a Z^a gate tuple (0.0 for every other gate)."""
    return float(g[3]) if len(g) > 3 else 0.0

SEED_BASE = 230310788

# The six Pauli-axis permutations as H/S words (circuit order) ...
_PERM_WORDS = [[], [H], [S], [H, S, H], [H, S], [S, H]]
# ... times the four Paulis give the 24 one-qubit Cliffords (mod phase).
_PAULI_WORDS = [[], [X], [Y], [Z]]
C1_WORDS = [p + q for p in _PERM_WORDS for q in _PAULI_WORDS]

# Double-coset representatives of C2 modulo C1 x C1 and their sizes.
_C2_CLASS_SIZES = np.array([576, 5184, 5184, 576], dtype=np.float64)


@dataclass
class Circuit:
    n_qubits: int
    gates: list = field(default_factory=list)   # (op, q0, q1) or (ZPOW, q, -1, a)

    def add(self, op, q0, q1=-1):
        self.gates.append((int(op), int(q0), int(q1)))

    def add_zpow(self, q, a):
        self.gates.append((ZPOW, int(q), -1, float(a)))

    @property
    def n_t(self):
        """Number of T, T^dagger and Z^a gates."""
        return sum(1 for g in self.gates if g[0] in (T, TDG, ZPOW))

    def as_array(self):
        """(n_gates, 3) int32 array of (op, q0, q1); exponents dropped."""
        if not self.gates:
            return np.zeros((0, 3), dtype=np.int32)
        return np.asarray([g[:3] for g in self.gates], dtype=np.int32)

    def params(self):
        """(n_gates,) float64 array of Z^a exponents (0 for other gates)."""
        return np.asarray([gate_param(g) for g in self.gates], dtype=np.float64)


@dataclass
class Region:
    full: list            # qubits inside the region for the whole circuit
    boundary: int         # qubit whose window [t_a, t_b) joins the region
    t_a: int
    t_b: int
    t_qubits: list        # qubits that may carry T gates
    n_t: int


@dataclass
class Workload:
    name: str
    circuit: Circuit
    cuts: list            # (qubit, gate_index): cut before gate_index on qubit
    marginal: list        # output qubits of the marginal, bit j = marginal[j]
    zstrings: list        # lists of qubits
    shots: int
    seed: int
    regions: list = field(default_factory=list)


def random_c1_word(rng):
    return list(C1_WORDS[rng.integers(24)])


def random_c2_word(rng, a, b):
    """Gate list of a uniformly random two-qubit Clifford on (a, b)."""
    cls = rng.choice(4, p=_C2_CLASS_SIZES / _C2_CLASS_SIZES.sum())
    out = []
    for q in (a, b):
        out += [(g, q, -1) for g in random_c1_word(rng)]
    core = [[], [(CX, a, b)], [(CX, a, b), (CX, b, a)],
            [(CX, a, b), (CX, b, a), (CX, a, b)]][cls]
    out += core
    for q in (a, b):
        out += [(g, q, -1) for g in random_c1_word(rng)]
    return out


def _frag_of(q, layer, regions):
    for i, r in enumerate(regions):
        if q in r.full:
            return i + 1
        if q == r.boundary and r.t_a <= layer < r.t_b:
            return i + 1
    return 0


def brickwork_star(n, depth, regions, seed):
    """Brickwork of random C2 elements with the star partition fixed first.

    At each layer the qubits are grouped by the fragment they belong to
    (body or a region); within each group consecutive members (in qubit
    order) are paired, alternating the pairing parity between layers.  So a
    region never splits the body's chain, and no gate straddles fragments.
    Returns ``(circuit, cuts)``; the cuts are the two wire cuts per region on
    its boundary qubit, at the first gate of layers t_a and t_b.
    """
    rng = np.random.default_rng(seed)
    # T positions: per region, n_t distinct (layer, qubit) slots.
    t_slots = set()
    for r in regions:
        cands = []
        for layer in range(depth):
            for q in r.t_qubits:
                if q == r.boundary and not (r.t_a <= layer < r.t_b):
                    continue
                cands.append((layer, q))
        pick = rng.choice(len(cands), size=min(r.n_t, len(cands)), replace=False)
        for i in pick:
            t_slots.add(cands[int(i)])
    c = Circuit(n)
    cuts = []
    for layer in range(depth):
        for r in regions:
            if layer in (r.t_a, r.t_b):
                cuts.append((r.boundary, len(c.gates)))
        groups = {}
        for q in range(n):
            groups.setdefault(_frag_of(q, layer, regions), []).append(q)
        pairs = []
        for members in groups.values():
            for j in range(layer % 2, len(members) - 1, 2):
                pairs.append((members[j], members[j + 1]))
        for a, b in sorted(pairs):
            c.gates += random_c2_word(rng, a, b)
        for q in range(n):
            if (layer, q) in t_slots:
                c.add(T, q)
    return c, cuts


def zstrings_for(n, count, rng, max_weight=8):
    out = []
    for _ in range(count):
        w = int(rng.integers(1, max_weight + 1))
        out.append(sorted(int(q) for q in rng.choice(n, size=min(w, n), replace=False)))
    return out


def _pick_marginal(rng, body_qubits, per_region, n_body):
    return per_region + sorted(int(q) for q in rng.choice(body_qubits, size=n_body, replace=False))


def small_star(n=8, depth=6, region_full=(0, 1), boundary=2, window=(2, 4),
               n_t=1, marginal=None, shots=1024, seed=1, n_z=8):
    """A small star-shaped workload (oracle-sized; used for parity cases)."""
    reg = Region(list(region_full), boundary, window[0], window[1],
                 list(region_full), n_t)
    c, cuts = brickwork_star(n, depth, [reg], seed)
    rng = np.random.default_rng(seed + 7)
    if marginal is None:
        body = [q for q in range(n) if q not in region_full]
        marginal = list(region_full[:2]) + sorted(int(q) for q in rng.choice(body, size=min(2, len(body)), replace=False))
    return Workload(f"star{n}x{depth}", c, cuts, list(marginal),
                    zstrings_for(n, n_z, rng, 4), shots, seed, [reg])


def config1():
    """16 qubits, 12 brickwork layers, 2 T on qubits 0-3, 2 cuts: 12q + 6q."""
    seed = SEED_BASE + 1
    reg = Region([0, 1, 2, 3, 4], 5, 4, 8, [0, 1, 2, 3], 2)
    c, cuts = brickwork_star(16, 12, [reg], seed)
    rng = np.random.default_rng(seed + 1)
    return Workload("config1", c, cuts, [0, 1, 2, 3, 12, 13, 14, 15],
                    zstrings_for(16, 16, rng, 8), 4096, seed, [reg])


def config2():
    """100 qubits, depth 20, two 9-wire NC regions with 5 T each, 4 cuts."""
    seed = SEED_BASE + 2
    rng = np.random.default_rng(seed + 1)
    ta1 = int(rng.integers(3, 8)); tb1 = ta1 + int(rng.integers(4, 8))
    ta2 = int(rng.integers(3, 8)); tb2 = ta2 + int(rng.integers(4, 8))
    r1 = Region(list(range(0, 8)), 8, ta1, tb1, list(range(0, 8)), 5)
    r2 = Region(list(range(92, 100)), 91, ta2, tb2, list(range(92, 100)), 5)
    c, cuts = brickwork_star(100, 20, [r1, r2], seed)
    body = [q for q in range(100) if q not in r1.full + r2.full]
    marg = _pick_marginal(rng, body, [0, 1, 2, 3, 92, 93, 94, 95], 4)
    return Workload("config2", c, cuts, marg, zstrings_for(100, 64, rng, 8),
                    10_000, seed, [r1, r2])


def config3():
    """500 qubits, depth 30, 4 regions of 1 full qubit + 1 boundary, 8 cuts."""
    seed = SEED_BASE + 3
    rng = np.random.default_rng(seed + 1)
    regs = []
    for i, q in enumerate([0, 130, 260, 390]):
        ta = int(rng.integers(4, 12)); tb = ta + int(rng.integers(6, 12))
        regs.append(Region([q], q + 1, ta, tb, [q, q + 1], 4))
    c, cuts = brickwork_star(500, 30, regs, seed)
    body = [q for q in range(500) if q not in (0, 130, 260, 390)]
    marg = _pick_marginal(rng, body, [0, 130, 260, 390], 12)
    return Workload("config3", c, cuts, marg, [], 1 << 14, seed, regs)


def _random_star(rng, n, depth, n_regions, n_t_total, max_width=10, min_depth_margin=2):
    """A random star workload: n_regions NC regions of width <= max_width."""
    regs = []
    used = set()
    starts = sorted(rng.choice(np.arange(0, n - max_width - 1, max_width + 2),
                               size=n_regions, replace=False))
    t_left = n_t_total
    for i, s0 in enumerate(starts):
        w = int(rng.integers(1, max_width))          # full qubits; +1 boundary
        full = list(range(int(s0), int(s0) + w))
        b = int(s0) + w
        ta = int(rng.integers(min_depth_margin, max(min_depth_margin + 1, depth // 2)))
        tb = int(min(depth - min_depth_margin, ta + rng.integers(2, max(3, depth // 2))))
        nt = t_left // (n_regions - i) if i < n_regions - 1 else t_left
        nt = max(1, nt)
        t_left -= nt
        regs.append(Region(full, b, ta, tb, full, nt))
        used.update(full + [b])
    return regs


def config4(n_circuits=256, seed_offset=0):
    """Many-circuit batch: n ~ U[50,300], depth ~ U[10,40], 1-3 regions."""
    seed = SEED_BASE + 4 + seed_offset
    rng = np.random.default_rng(seed)
    out = []
    for ci in range(n_circuits):
        n = int(rng.integers(50, 301))
        depth = int(rng.integers(10, 41))
        nreg = int(rng.integers(1, 4))
        nt = int(rng.integers(max(2, nreg), 13))
        regs = _random_star(rng, n, depth, nreg, nt)
        c, cuts = brickwork_star(n, depth, regs, int(rng.integers(1 << 31)))
        nc_q = [q for r in regs for q in r.full]
        body = [q for q in range(n) if q not in nc_q]
        per_reg = [r.full[0] for r in regs]
        marg = per_reg + sorted(int(q) for q in rng.choice(body, size=10 - len(per_reg), replace=False))
        out.append(Workload(f"config4_{ci}", c, cuts, marg, [], 4096,
                            seed * 1000 + ci, regs))
    return out


def config5_circuit(rng, n_lo=50, n_hi=401, t_lo=4, t_hi=41, max_regions=4):
    """One circuit of the learned-cut population (no intended cut set used)."""
    n = int(rng.integers(n_lo, n_hi))
    depth = int(rng.integers(10, 41))
    nreg = int(rng.integers(1, max_regions + 1))
    nt = int(rng.integers(max(t_lo, nreg), t_hi))
    regs = _random_star(rng, n, depth, nreg, nt, max_width=6)
    c, cuts = brickwork_star(n, depth, regs, int(rng.integers(1 << 31)))
    return c, cuts, regs


# Clifford-angle rotations as gate words (circuit order), up to global phase:
# R_z(k pi/2) = S^k, R_y(k pi/2), R_x(k pi/2) = H R_z(k pi/2) H.
RZ_WORDS = [[], [S], [Z], [SDG]]
RY_WORDS = [[], [Z, H], [Y], [H, Z]]
RX_WORDS = [[], [H, S, H], [X], [H, SDG, H]]


def _inject(rng, c, n_t, zpow):
    """Insert n_t non-Clifford gates at uniformly random (position, qubit):
    T or T^dagger, or Z^a with a uniform in (0, 2) off the multiples of 1/2."""
    for _ in range(n_t):
        pos = int(rng.integers(len(c.gates) + 1))
        q = int(rng.integers(c.n_qubits))
        if zpow:
            a = float(rng.uniform(0.02, 0.48)) + 0.5 * int(rng.integers(4))
            c.gates.insert(pos, (ZPOW, q, -1, a))
        else:
            c.gates.insert(pos, (T if rng.random() < 0.5 else TDG, q, -1))


def hwea(n, rounds=5, n_t=1, seed=SEED_BASE + 6, marginal=10, n_z=0, shots=4096, zpow=False):
    """Near-Clifford hardware-efficient ansatz (Sec. VI-B): per round a layer
    of one-qubit rotations R_y R_z, a linear chain of CX entanglers and a
    second rotation layer, every angle a multiple of pi/2 (a Clifford ansatz,
    Sec. IV-B), with n_t non-Clifford gates injected at random places.  No
    cut set: the cut search chooses one."""
    rng = np.random.default_rng(seed)
    c = Circuit(n)

    def rotations():
        for q in range(n):
            for op in RY_WORDS[int(rng.integers(4))] + RZ_WORDS[int(rng.integers(4))]:
                c.add(op, q)

    for _ in range(rounds):
        rotations()
        for q in range(n - 1):
            c.add(CX, q, q + 1)
        rotations()
    _inject(rng, c, n_t, zpow)
    marg = sorted(int(q) for q in rng.choice(n, size=min(marginal, n), replace=False))
    return Workload(f"hwea{n}x{rounds}", c, None, marg, zstrings_for(n, n_z, rng), shots, seed)


def sk_qaoa(n, rounds=1, n_t=1, seed=SEED_BASE + 7, marginal=10, n_z=0, shots=4096, zpow=False):
    """Near-Clifford MaxCut QAOA on the Sherrington-Kirkpatrick model
    (Sec. VI-B): |+>^n, then per round exp(-i gamma J_ab Z_a Z_b) on every
    pair (all-to-all, J_ab = +-1, as CX R_z CX) and the mixer R_x(beta) on
    every qubit, gamma and beta multiples of pi/4 so that every rotation is
    Clifford; n_t non-Clifford gates injected at random places."""
    rng = np.random.default_rng(seed)
    c = Circuit(n)
    for q in range(n):
        c.add(H, q)
    for _ in range(rounds):
        g = int(rng.integers(1, 4))             # gamma = g pi/4
        b = int(rng.integers(1, 4))             # beta = b pi/4
        for a in range(n):
            for q in range(a + 1, n):
                k = (g * (1 if rng.random() < 0.5 else -1)) % 4
                c.add(CX, a, q)
                for op in RZ_WORDS[k]:
                    c.add(op, q)
                c.add(CX, a, q)
        for q in range(n):
            for op in RX_WORDS[b]:
                c.add(op, q)
    _inject(rng, c, n_t, zpow)
    marg = sorted(int(q) for q in rng.choice(n, size=min(marginal, n), replace=False))
    return Workload(f"skqaoa{n}x{rounds}", c, None, marg, zstrings_for(n, n_z, rng), shots, seed)


def random_clifford_circuit(n, n_gates, seed, t_count=0):
    """Unstructured random circuit over the full gate set (oracle pins)."""
    rng = np.random.default_rng(seed)
    c = Circuit(n)
    ops1 = [H, S, SDG, X, Y, Z]
    for _ in range(n_gates):
        if n > 1 and rng.random() < 0.4:
            a, b = (int(v) for v in rng.choice(n, size=2, replace=False))
            c.add([CX, CZ][int(rng.integers(2))], a, b)
        else:
            c.add(ops1[int(rng.integers(len(ops1)))], int(rng.integers(n)))
    for _ in range(t_count):
        pos = int(rng.integers(len(c.gates) + 1))
        c.gates.insert(pos, (T if rng.random() < 0.5 else TDG, int(rng.integers(n)), -1))
    return c


def tree_circuit(parents, gates_per_block, n_t, seed, width=3):
    """Blocks of ``width`` wires joined in a tree: block b (b >= 1) hangs below
    block ``parents[b-1]``.  Each child block's first wire takes one CX from
    its parent block's second wire and is cut right after it, so the
    fragments follow the tree (a chain, or branches of any shape).  Returns
    (circuit, cuts); T/TDG gates are placed after the cuts."""
    rng = np.random.default_rng(seed)
    nb = len(parents) + 1
    c = Circuit(nb * width)
    ops1 = [H, S, SDG, X, Y, Z]
    child_first = {b * width for b in range(1, nb)}

    def fill(count, before_cuts):
        for _ in range(count):
            b = int(rng.integers(nb))
            qs = [b * width + i for i in range(width)]
            if rng.random() < 0.45:
                # before the cuts a child's first wire stays out of its block
                pool = qs[1:] if (before_cuts and qs[0] in child_first) else qs
                a, t = (int(v) for v in rng.choice(pool, size=2, replace=False))
                c.add([CX, CZ][int(rng.integers(2))], a, t)
            else:
                c.add(ops1[int(rng.integers(len(ops1)))], int(rng.choice(qs)))

    for q in range(c.n_qubits):
        c.add(H, q)
    fill(gates_per_block * nb // 2, True)
    for b, p in enumerate(parents, start=1):
        c.add(CX, p * width + 1, b * width)
    cuts = [(b * width, len(c.gates)) for b in range(1, nb)]
    start = len(c.gates)
    fill(gates_per_block * nb // 2, False)
    for _ in range(n_t):
        pos = int(rng.integers(start, len(c.gates) + 1))
        c.gates.insert(pos, (T if rng.random() < 0.5 else TDG, int(rng.integers(c.n_qubits)), -1))
    return c, cuts


def t_to_s(circuit):
    """Replace every T by S and TDG by SDG (the circuit becomes Clifford)."""
    c = Circuit(circuit.n_qubits)
    for g in circuit.gates:
        c.gates.append(({T: S, TDG: SDG}.get(g[0], g[0]),) + tuple(g[1:]))
    return c


def random_distributions(n_variants, n_bits, seed, sparsity=0.5):
    """Random per-variant probability tables (rows sum to 1), float64.

    Synthetic fragment results of the right shape, used to drive the fold and
    recombination stages on their own at full size.
    """
    rng = np.random.default_rng(seed)
    p = rng.random((n_variants, 1 << n_bits))
    p[rng.random(p.shape) < sparsity] = 0.0
    p[:, 0] += 1e-3
    return p / p.sum(axis=1, keepdims=True)
