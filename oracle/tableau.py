"""ORACLE (test infrastructure): naive CHP stabilizer tableau and its outcome space.

Clifford circuits are simulable in polynomial time by tracking how Pauli
strings are conjugated (Gottesman-Knill, Sec. II-C; the CHP tableau of
Aaronson and Gottesman cited in Sec. III-B).  Rows 0..n-1 are destabilizers,
rows n..2n-1 stabilizers; row i is (-1)^r[i] prod_j P(x[i,j], z[i,j]) with
P(1,1) = Y.  One byte per bit; every update is a column operation written out
from the CHP rules.

The Z-measurement distribution of a stabilizer state is uniform on an affine
subspace, and every Pauli expectation is -1, 0 or +1 (Sec. IX).  The affine
space is found by the textbook route: full Gaussian elimination of the
stabilizer X-block with phase-tracked row products; the rows left with zero
X part are Z-type constraints z.x = r; their solution set is x0 + span(D)
with D the X-parts of the eliminated rows.  Restricted to a measured wire list
A this is returned canonically: B = RREF of D|A (pivot = lowest A-index, rows
ordered by pivot), off = x0|A with every pivot bit cleared by B.
"""
from __future__ import annotations

import numpy as np

from workloads import H, S, SDG, X, Y, Z, CX, CZ, T, TDG, ZPOW, gate_param


class Tableau:
    """Byte-per-bit CHP tableau of n qubits, initialised to |0...0>."""

    def __init__(self, n):
        self.n = n
        self.x = np.zeros((2 * n, n), np.uint8)
        self.z = np.zeros((2 * n, n), np.uint8)
        self.r = np.zeros(2 * n, np.uint8)
        for i in range(n):
            self.x[i, i] = 1          # destabilizer i = X_i
            self.z[n + i, i] = 1      # stabilizer i = Z_i

    def copy(self):
        t = Tableau.__new__(Tableau)
        t.n, t.x, t.z, t.r = self.n, self.x.copy(), self.z.copy(), self.r.copy()
        return t

    # --- gate rules (conjugation of every row) -----------------------------
    def h(self, a):
        xa, za = self.x[:, a].copy(), self.z[:, a].copy()
        self.r ^= xa & za
        self.x[:, a], self.z[:, a] = za, xa

    def s(self, a):
        xa, za = self.x[:, a], self.z[:, a]
        self.r ^= xa & za
        self.z[:, a] = za ^ xa

    def sdg(self, a):
        xa, za = self.x[:, a], self.z[:, a]
        self.r ^= xa & (za ^ 1)
        self.z[:, a] = za ^ xa

    def pauli_x(self, a):
        self.r ^= self.z[:, a]

    def pauli_y(self, a):
        self.r ^= self.x[:, a] ^ self.z[:, a]

    def pauli_z(self, a):
        self.r ^= self.x[:, a]

    def cx(self, c, t):
        xc, zc = self.x[:, c].copy(), self.z[:, c].copy()
        xt, zt = self.x[:, t].copy(), self.z[:, t].copy()
        self.r ^= xc & zt & (xt ^ zc ^ 1)
        self.x[:, t] = xt ^ xc
        self.z[:, c] = zc ^ zt

    def cz(self, a, b):
        xa, za = self.x[:, a].copy(), self.z[:, a].copy()
        xb, zb = self.x[:, b].copy(), self.z[:, b].copy()
        self.r ^= xa & xb & (za ^ zb)
        self.z[:, a] = za ^ xb
        self.z[:, b] = zb ^ xa

    def apply(self, op, a, b=-1, param=0.0):
        if op == ZPOW:
            # Z^a = (Z^{1/2})^{2a} = S^{2a}: Clifford exactly when 2a is an
            # integer (e^{i pi a} in {1, i, -1, -i}), Sec. II-C
            k = 2.0 * param
            if k != np.floor(k):
                raise ValueError("Z^a with 2a not an integer is not a Clifford gate")
            for _ in range(int(k) % 4):
                self.s(a)
        elif op == H:
            self.h(a)
        elif op == S:
            self.s(a)
        elif op == SDG:
            self.sdg(a)
        elif op == X:
            self.pauli_x(a)
        elif op == Y:
            self.pauli_y(a)
        elif op == Z:
            self.pauli_z(a)
        elif op == CX:
            self.cx(a, b)
        elif op == CZ:
            self.cz(a, b)
        elif op in (T, TDG):
            raise ValueError("T is not a Clifford gate")
        else:
            raise ValueError(f"unknown gate {op}")

    def run(self, gates):
        for g in gates:
            self.apply(g[0], g[1], g[2], gate_param(g))
        return self


def g_sum(x1, z1, x2, z2):
    """Sum over qubits of the exponent of i picked up by P1*P2 (per-qubit g)."""
    x1 = x1.astype(np.int64); z1 = z1.astype(np.int64)
    x2 = x2.astype(np.int64); z2 = z2.astype(np.int64)
    g = np.where((x1 == 1) & (z1 == 1), z2 - x2,
        np.where((x1 == 1) & (z1 == 0), z2 * (2 * x2 - 1),
        np.where((x1 == 0) & (z1 == 1), x2 * (1 - 2 * z2), 0)))
    return g.sum(axis=-1)


def row_product_into(x, z, r, targets, src):
    """rowsum: multiply row ``src`` into each row of ``targets`` (in place).

    The phase of the product of two commuting rows is 2r_h + 2r_i + sum g,
    which must be 0 or 2 mod 4.
    """
    if len(targets) == 0:
        return
    e = (2 * r[targets].astype(np.int64) + 2 * int(r[src])
         + g_sum(x[src][None, :], z[src][None, :], x[targets], z[targets])) % 4
    assert np.all((e == 0) | (e == 2)), "row product of anticommuting rows"
    r[targets] = (e // 2).astype(np.uint8)
    x[targets] ^= x[src][None, :]
    z[targets] ^= z[src][None, :]


def gf2_rref(rows):
    """RREF over GF(2) of a list of ints (bit j = column j), pivot = lowest bit.

    Returns (basis rows ordered by pivot ascending, pivots).
    """
    rows = [int(v) for v in rows if v]
    basis, pivots = [], []
    for j in range(max((v.bit_length() for v in rows), default=0)):
        sel = next((i for i, v in enumerate(rows) if (v >> j) & 1), None)
        if sel is None:
            continue
        p = rows.pop(sel)
        rows = [v ^ p if (v >> j) & 1 else v for v in rows]
        basis = [v ^ p if (v >> j) & 1 else v for v in basis]
        basis.append(p)
        pivots.append(j)
        rows = [v for v in rows if v]
    order = sorted(range(len(basis)), key=lambda i: pivots[i])
    return [basis[i] for i in order], [pivots[i] for i in order]


def support(tab):
    """Affine support x0 + span(D) of the state's Z-basis distribution.

    Returns (x0 as uint8 vector of length n, D as (rank, n) uint8 matrix).
    """
    n = tab.n
    x, z, r = tab.x[n:].copy(), tab.z[n:].copy(), tab.r[n:].copy()
    rank = 0
    for col in range(n):
        piv = next((i for i in range(rank, n) if x[i, col]), None)
        if piv is None:
            continue
        if piv != rank:
            for arr in (x, z, r):
                arr[[piv, rank]] = arr[[rank, piv]]
        tgt = np.array([h for h in range(n) if h != rank and x[h, col]], dtype=np.int64)
        row_product_into(x, z, r, tgt, rank)
        rank += 1
    # Rows rank..n-1 are Z-type: (-1)^r Z^z, i.e. constraints z.x = r.
    zrows = [(int(''.join(map(str, z[h][::-1])), 2) if n else 0) | (int(r[h]) << n)
             for h in range(rank, n)]
    # Solve by RREF of the augmented rows; free variables are 0.
    aug, piv = gf2_rref(zrows)
    x0 = np.zeros(n, np.uint8)
    for row, p in zip(aug, piv):
        assert p < n, "inconsistent Z constraints"
        x0[p] = (row >> n) & 1
    return x0, x[:rank].copy()


def outcome_space(tab, A):
    """Canonical (off, B, rho) of Z-measuring wires A (bit j of y = wire A[j])."""
    x0, D = support(tab)
    def proj(vec):
        return sum(int(vec[a]) << j for j, a in enumerate(A))
    B, piv = gf2_rref([proj(d) for d in D])
    off = proj(x0)
    for b, p in zip(B, piv):
        if (off >> p) & 1:
            off ^= b
    return off, B, len(B)


def z_expectation(tab, wires, supp=None):
    """<Z_wires> of the state: (-1)^{mask.x0} if mask is orthogonal to D, else 0.

    ``supp`` may pass a precomputed ``support(tab)``."""
    x0, D = support(tab) if supp is None else supp
    mask = np.zeros(tab.n, np.uint8)
    for w in wires:
        mask[w] ^= 1
    if D.size and np.any((D.astype(np.int64) @ mask.astype(np.int64)) % 2):
        return 0.0
    return -1.0 if int(mask.astype(np.int64) @ x0.astype(np.int64)) % 2 else 1.0


def exact_distribution(off, B, nbits):
    """p(y) = 2^-rho on off + span(B), as a dense float64 vector."""
    pts = np.array([off], dtype=np.int64)
    for b in B:
        pts = np.concatenate([pts, pts ^ b])
    p = np.zeros(1 << nbits)
    p[pts] = 1.0 / len(pts)
    return p


def tableau_bits(tab):
    """Export as uint8 [2n, 2n+1]: x_0..x_{n-1}, z_0..z_{n-1}, r."""
    return np.concatenate([tab.x, tab.z, tab.r[:, None]], axis=1)
