"""Pins of the oracle against facts fixed outside itself (no GPU).

Each test checks the oracle against brute force, a closed form, a published
known-answer vector or an invariant, never against a retyped copy of itself.
"""
import itertools
import os

import numpy as np
import pytest

from workloads import (H, S, SDG, X, Y, Z, CX, CZ, T, TDG, ZPOW, Circuit, small_star, config1,
                       random_clifford_circuit, t_to_s, brickwork_star, Region, hwea, sk_qaoa)
from workloads.circuits import C1_WORDS
from oracle import tableau as tb
from oracle import statevector as sv
from oracle.philox import philox4x32_10, shot_coeffs, shot_words
from oracle.pipeline import evaluate, evaluate_workload, brute_force, uncut_clifford, sample_counts

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# --- dense Pauli algebra (independent of the tableau rules) ---------------
_P1 = {(0, 0): np.eye(2), (1, 0): sv.MATS[X], (0, 1): sv.MATS[Z], (1, 1): sv.MATS[Y]}


def dense_pauli(xs, zs, r):
    m = np.array([[1.0 + 0j]])
    for q in reversed(range(len(xs))):          # qubit 0 = least significant
        m = np.kron(m, _P1[(int(xs[q]), int(zs[q]))])
    return m * (-1) ** int(r)


def dense_gate(n, op, a, b=-1):
    d = 1 << n
    U = np.zeros((d, d), complex)
    for i in range(d):
        e = np.zeros(d, complex); e[i] = 1
        U[:, i] = sv.apply(e, n, op, a, b)
    return U


def all_rows(n):
    rows = list(itertools.product([0, 1], repeat=2 * n))
    x = np.array([r[:n] for r in rows], np.uint8)
    z = np.array([r[n:] for r in rows], np.uint8)
    return x, z


@pytest.mark.parametrize("op,qs", [(H, (0,)), (S, (0,)), (SDG, (0,)), (X, (0,)), (Y, (0,)),
                                   (Z, (0,)), (CX, (0, 1)), (CX, (1, 0)), (CZ, (0, 1)),
                                   (H, (1,)), (S, (1,))])
def test_gate_rule_equals_dense_conjugation(op, qs):
    """Every CHP column update equals U P U^dagger for all 16 two-qubit Paulis and both signs."""
    n = 2
    x, z = all_rows(n)
    for r0 in (0, 1):
        t = tb.Tableau.__new__(tb.Tableau)
        t.n = n
        t.x, t.z = x.copy(), z.copy()
        t.r = np.full(len(x), r0, np.uint8)
        t.apply(op, *qs) if len(qs) == 2 else t.apply(op, qs[0])
        U = dense_gate(n, op, *qs)
        for i in range(len(x)):
            want = U @ dense_pauli(x[i], z[i], r0) @ U.conj().T
            got = dense_pauli(t.x[i], t.z[i], t.r[i])
            assert np.allclose(want, got), (op, qs, i, r0)


def test_gate_identities():
    c = random_clifford_circuit(5, 60, seed=3)
    t0 = tb.Tableau(5).run(c.gates)
    for seq in ([(S, 2, -1), (SDG, 2, -1)], [(H, 1, -1), (H, 1, -1)],
                [(CX, 0, 3), (CX, 0, 3)], [(S, 4, -1)] * 4, [(CZ, 1, 2), (CZ, 2, 1)]):
        t = t0.copy().run(seq)
        assert np.array_equal(tb.tableau_bits(t), tb.tableau_bits(t0))


def _bfs_clifford_count(n_qubits, gens):
    start = tb.Tableau(n_qubits)
    key = lambda t: tb.tableau_bits(t).tobytes()
    seen = {key(start)}
    frontier = [start]
    while frontier:
        nxt = []
        for t in frontier:
            for g in gens:
                u = t.copy(); u.apply(*g)
                kk = key(u)
                if kk not in seen:
                    seen.add(kk); nxt.append(u)
        frontier = nxt
    return len(seen)


def test_clifford_group_orders():
    """|C1| = 24 and |C2| = 11520 (mod phase: 2^{n^2+2n} prod_j (4^j - 1))."""
    assert _bfs_clifford_count(1, [(H, 0, -1), (S, 0, -1)]) == 24
    gens = [(H, 0, -1), (H, 1, -1), (S, 0, -1), (S, 1, -1), (CX, 0, 1), (CX, 1, 0)]
    assert _bfs_clifford_count(2, gens) == 2 ** 8 * 3 * 15 == 11520


def test_generator_c1_words_are_the_24_cliffords():
    keys = {tb.tableau_bits(tb.Tableau(1).run([(g, 0, -1) for g in w])).tobytes() for w in C1_WORDS}
    assert len(keys) == 24


def test_tableau_commutation_invariants():
    """Destabilizer i anticommutes with stabilizer i only; all others commute."""
    for seed in range(4):
        n = 7
        t = tb.Tableau(n).run(random_clifford_circuit(n, 80, seed).gates)
        x, z = t.x.astype(int), t.z.astype(int)
        gram = (x @ z.T + z @ x.T) % 2
        want = np.zeros((2 * n, 2 * n), int)
        for i in range(n):
            want[i, n + i] = want[n + i, i] = 1
        assert np.array_equal(gram, want)


@pytest.mark.parametrize("seed", range(6))
def test_outcome_space_matches_statevector(seed):
    """Z-probabilities on A are 2^-rho on off + span(B) and 0 elsewhere (brute force)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 9))
    c = random_clifford_circuit(n, 10 * n, seed + 100)
    A = [int(a) for a in rng.permutation(n)[: int(rng.integers(1, n + 1))]]
    t = tb.Tableau(n).run(c.gates)
    off, B, rho = tb.outcome_space(t, A)
    p = sv.marginal(sv.run(n, c.gates), n, A)
    assert np.allclose(p, tb.exact_distribution(off, B, len(A)), atol=1e-12)
    # canonical form: pivots ascending, fully reduced, off has no pivot bits
    piv = [(b & -b).bit_length() - 1 for b in B]
    assert piv == sorted(piv)
    for i, b in enumerate(B):
        for j, pj in enumerate(piv):
            assert ((b >> pj) & 1) == (i == j)
        assert not (off >> piv[i]) & 1
    for zs in [A[:1], A[:2], A]:
        assert abs(tb.z_expectation(t, zs) - sv.z_expectation(sv.run(n, c.gates), n, zs)) < 1e-12


def test_zpow_special_exponents():
    """Z^a = diag(1, e^{i pi a}) is the identity at a = 0 and 2, and the
    named gates of Sec. II-C at a = 1/2 (S), 1 (Z), -1/2 = 3/2 (S^dagger),
    1/4 (T) and -1/4 (T^dagger)."""
    for a in (0.0, 2.0, -4.0):
        assert np.allclose(sv.zpow_matrix(a), np.eye(2), atol=1e-15)
    for a, op in ((0.5, S), (1.0, Z), (-0.5, SDG), (1.5, SDG), (0.25, T), (-0.25, TDG), (2.25, T)):
        assert np.allclose(sv.zpow_matrix(a), sv.MATS[op], atol=1e-15), a


def _insert_zpow(c, exps, seed):
    rng = np.random.default_rng(seed)
    for a in exps:
        c.gates.insert(int(rng.integers(len(c.gates) + 1)), (ZPOW, int(rng.integers(c.n_qubits)), -1, float(a)))
    return c


@pytest.mark.parametrize("seed", range(4))
def test_clifford_zpow_tableau_matches_statevector(seed):
    """Z^a with 2a an integer is S^{2a}: the tableau's outcome space and
    Z-string values equal the dense statevector's (brute force), for
    exponents on both sides of zero and beyond one period."""
    n = 6
    c = _insert_zpow(random_clifford_circuit(n, 60, seed + 300), (0.5, 1.0, 1.5, 2.0, -0.5, 3.5, 7.0, -2.5), seed)
    A = [0, 2, 3, 5]
    t = tb.Tableau(n).run(c.gates)
    off, B, rho = tb.outcome_space(t, A)
    psi = sv.run(n, c.gates)
    assert np.allclose(sv.marginal(psi, n, A), tb.exact_distribution(off, B, len(A)), atol=1e-12)
    for zs in ([0], [1, 4], [0, 2, 3, 5]):
        assert abs(tb.z_expectation(t, zs) - sv.z_expectation(psi, n, zs)) < 1e-12
    with pytest.raises(ValueError):
        tb.Tableau(2).run([(ZPOW, 0, -1, 0.3)])


@pytest.mark.parametrize("seed", range(3))
def test_cut_identity_with_zpow(seed):
    """Non-Clifford Z^a (2a not an integer) inside the cut-out regions: the
    exact recombination equals the uncut statevector."""
    rng = np.random.default_rng(seed)
    w = small_star(n=9, depth=7, region_full=(0, 1, 2), boundary=3, window=(2, 5), n_t=3, seed=20 + seed)
    c = Circuit(w.circuit.n_qubits)
    for g in w.circuit.gates:       # every T becomes Z^a at the same place
        c.gates.append((ZPOW, g[1], -1, float(rng.uniform(-3, 3))) if g[0] == T else g)
    r = evaluate(c, w.cuts, w.marginal, w.zstrings, mode="exact")
    assert sum(not f.clifford for f in r.fragments) == 1
    bf, bz = brute_force(c, w.marginal, w.zstrings)
    assert np.abs(r.marginal - bf).max() < 1e-12
    assert np.abs(r.zexp - bz).max() < 1e-12


def test_paper_workload_generators():
    """HWEA and SK-QAOA (Sec. VI-B): with the injected gates removed the
    circuits are Clifford (the tableau accepts them) and the statevector of
    the Clifford ansatz has the affine-space distribution."""
    for w in (hwea(8, rounds=5, n_t=2), sk_qaoa(7, n_t=1), hwea(6, rounds=3, n_t=2, zpow=True),
              sk_qaoa(6, n_t=2, zpow=True)):
        c = w.circuit
        assert sum(g[0] in (T, TDG, ZPOW) for g in c.gates) == c.n_t > 0
        cl = Circuit(c.n_qubits, [g for g in c.gates if g[0] not in (T, TDG, ZPOW)])
        t = tb.Tableau(cl.n_qubits).run(cl.gates)
        A = list(range(cl.n_qubits))
        off, B, rho = tb.outcome_space(t, A)
        p = sv.marginal(sv.run(cl.n_qubits, cl.gates), cl.n_qubits, A)
        assert np.allclose(p, tb.exact_distribution(off, B, len(A)), atol=1e-12)
    # SK-QAOA is all-to-all: every pair interacts
    c = sk_qaoa(9).circuit
    pairs = {tuple(sorted(g[1:3])) for g in c.gates if g[0] == CX}
    assert len(pairs) == 9 * 8 // 2


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    for r in rows:
        v = [int(s, 16) for s in r]
        out = philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


@pytest.mark.parametrize("w", [small_star(), small_star(n=9, depth=7, region_full=(0, 1, 2),
                                                     boundary=3, window=(2, 5), n_t=2, seed=5),
                               small_star(n=6, depth=5, region_full=(0,), boundary=1,
                                          window=(1, 3), n_t=1, seed=9)])
def test_cut_identity_small(w):
    r = evaluate_workload(w, mode="exact")
    bf, bz = brute_force(w.circuit, w.marginal, w.zstrings)
    assert np.abs(r.marginal - bf).max() < 1e-12
    assert np.abs(r.zexp - bz).max() < 1e-12
    assert abs(r.marginal.sum() - 1) < 1e-12


def test_cut_identity_config1():
    """16 qubits: exact-mode recombined marginal equals the uncut statevector."""
    w = config1()
    r = evaluate_workload(w, mode="exact")
    assert [f.n for f in r.fragments] == [6, 12]
    assert [f.n_variants for f in r.fragments] == [12, 12]
    bf, bz = brute_force(w.circuit, w.marginal, w.zstrings)
    assert np.abs(r.marginal - bf).max() < 1e-12
    assert np.abs(r.zexp - bz).max() < 1e-12


@pytest.mark.parametrize("seed", range(5))
def test_cut_set_invariance_random_cuts(seed):
    """Any valid cut set (random wires and times, any topology) gives the uncut result."""
    rng = np.random.default_rng(seed)
    n = 5
    c = random_clifford_circuit(n, 30, seed, t_count=2)
    marg = [0, 2, 4]
    z = [[0, 1], [3], [1, 2, 4]]
    bf, bz = brute_force(c, marg, z)
    tried = 0
    while tried < 2:
        ncut = int(rng.integers(1, 4))
        cuts = [(int(rng.integers(n)), int(rng.integers(1, len(c.gates)))) for _ in range(ncut)]
        try:
            r = evaluate(c, cuts, marg, z, mode="exact")
        except ValueError:
            continue
        tried += 1
        assert np.abs(r.marginal - bf).max() < 1e-12
        assert np.abs(r.zexp - bz).max() < 1e-12


def test_t_to_s_large_n():
    """With every T replaced by S, the cut result equals one uncut tableau's closed form."""
    regs = [Region([0, 1, 2], 3, 3, 7, [0, 1, 2], 3), Region([36, 37], 35, 4, 8, [36, 37], 2)]
    c, cuts = brickwork_star(38, 10, regs, seed=11)
    c = t_to_s(c)
    marg = [0, 1, 36, 37, 10, 20, 30]
    zs = [[0, 5, 36], [12, 13], [1, 2, 3, 4, 37]]
    r = evaluate(c, cuts, marg, zs, mode="exact")
    cf, cz = uncut_clifford(c, marg, zs)
    assert len(r.fragments) == 3
    assert np.abs(r.marginal - cf).max() < 1e-12
    assert np.abs(r.zexp - cz).max() < 1e-12


def test_sampling_is_uniform_on_the_affine_space():
    rng = np.random.default_rng(0)
    n = 8
    c = random_clifford_circuit(n, 60, 21)
    A = list(range(n))
    t = tb.Tableau(n).run(c.gates)
    off, B, rho = tb.outcome_space(t, A)
    shots = 20000
    counts = sample_counts(off, B, len(A), shots, 3, 1, 0, 77, 88)
    exact = tb.exact_distribution(off, B, len(A))
    assert counts.sum() == shots
    assert np.all(counts[exact == 0] == 0)
    e = shots * exact[exact > 0]
    chi2 = float(((counts[exact > 0] - e) ** 2 / e).sum())
    dof = (1 << rho) - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof) + 10


def test_sampled_mode_converges_and_normalises():
    """Exact mode sums to 1 exactly.  Sampled mode does only up to shot noise
    here: the NC fragment both receives and emits a cut wire, so its sampled
    expectations at the emitted cut differ between preparations and the
    mu-weighted sum over preparations no longer cancels exactly."""
    w = small_star(shots=1 << 15)
    rs = evaluate_workload(w, mode="sampled")
    re = evaluate_workload(w, mode="exact")
    assert abs(re.marginal.sum() - 1) < 1e-12
    assert abs(rs.marginal.sum() - 1) < 8 / np.sqrt(w.shots)
    assert np.abs(rs.marginal - re.marginal).max() < 8 / np.sqrt(w.shots)


def test_shot_words_keying():
    a = shot_words(8, 1, 2, 3, 10, 20)
    b = shot_words(8, 1, 2, 3, 10, 21)
    c = shot_words(8, 2, 2, 3, 10, 20)
    assert len(set(a.tolist())) == 8 and not np.array_equal(a, b) and not np.array_equal(a, c)


def test_shot_words_layout():
    """Shot 4k+j is output word j of the generator at counter (k, v, f, c);
    a ragged shot count takes a prefix (the counter layout is this
    implementation's choice: the paper fixes none)."""
    w = shot_words(11, 5, 6, 7, 0xA, 0xB)
    for k in range(3):
        out = philox4x32_10(k, 5, 6, 7, 0xA, 0xB)
        for j in range(4):
            if 4 * k + j < 11:
                assert int(w[4 * k + j]) == int(out[j])
    assert np.array_equal(shot_words(7, 5, 6, 7, 0xA, 0xB), w[:7])


@pytest.mark.parametrize("rank,per_word", [(0, 4), (5, 4), (8, 4), (9, 2), (16, 2), (17, 1), (24, 1)])
def test_shot_coeffs_layout(rank, per_word):
    """A word serves four shots at rank <= 8 (bytes, low byte first), two at
    rank <= 16 (half words), one above; each shot keeps its low rank bits.
    Checked against the generator's raw output words, shot by shot."""
    n = 37
    c = shot_coeffs(n, rank, 5, 6, 7, 0xA, 0xB)
    width = 32 // per_word
    for t in range(n):
        widx = t // per_word
        word = int(philox4x32_10(widx // 4, 5, 6, 7, 0xA, 0xB)[widx % 4])
        field = (word >> (width * (t % per_word))) & ((1 << width) - 1)
        assert int(c[t]) == field & ((1 << rank) - 1), (t, rank)
