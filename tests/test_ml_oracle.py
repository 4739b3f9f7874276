"""Pins of the maximum-likelihood correction oracle (Sec. V-C) against facts
fixed outside it (no GPU): the identity channel's Choi operator in closed
form, positivity of every exactly evaluated fragment (which fails if the
input transpose is dropped), trace preservation, the simplex projection on a
worked case and against brute-force optimality, the correction as the
nearest physical model (first-order optimality against random physical
models) and its effect on a sampled workload (no negative
quasi-probabilities left, closer to the uncut statevector).
"""
import numpy as np
import pytest

from workloads import Workload, tree_circuit, small_star
from oracle import statevector as sv
from oracle.cutting import Fragment, fold, fragment_circuit, recombine
from oracle.mlcorrect import (choi_blocks, tensor_from_choi, project_simplex, ml_correct,
                              is_physical, slot_is_input)
from oracle.pipeline import evaluate, brute_force


def exact_tensor(frag):
    """T_f of a fragment from exact statevector distributions of its variants."""
    dists = [sv.marginal(sv.run(frag.n, frag.variant_gates(v)), frag.n, frag.A)
             for v in range(frag.n_variants)]
    return fold(frag, dists)


def test_identity_channel_closed_form():
    """A bare wire with one input and one output: T(P_in, P_out) = Tr[P_out P_in]
    = 2 delta, and the Choi operator is 2 |Phi+><Phi+| (eigenvalues 2, 0, 0, 0)."""
    f = Fragment(wires=[(0, 1)], gates=[], qin=[(0, 0)], qout=[(1, 0)], marg=[], slots=[0, 1])
    T = exact_tensor(f)
    want = np.zeros((1, 16))
    for p in range(4):
        want[0, p + 4 * p] = 2.0
    assert np.abs(T - want).max() < 1e-12
    J = choi_blocks(f, T)[0]
    phi = np.zeros(4); phi[0] = phi[3] = 2 ** -0.5
    assert np.abs(J - 2 * np.outer(phi, phi)).max() < 1e-12
    assert np.allclose(np.linalg.eigvalsh(J), [0, 0, 0, 2], atol=1e-12)


def _fragments_with_inputs():
    out = []
    for parents, n_t, seed in (([0, 1], 2, 3), ([0, 0], 1, 5), ([0, 1, 1], 2, 7)):
        c, cuts = tree_circuit(parents, 10, n_t, seed=seed)
        frags, _ = fragment_circuit(c, cuts, [0, 2, c.n_qubits - 1])
        out += frags
    return out


def test_exact_fragments_are_physical_and_need_the_input_transpose():
    """Every exactly evaluated fragment (Clifford or not) is a CP,
    trace-preserving instrument: all Choi blocks PSD, sum_o Tr_out J_o = I on
    the inputs.  For a unitary one-wire fragment the Choi operator is
    maximally entangled, and without the transpose at the input it has a
    negative eigenvalue (the plausible mistake this pins)."""
    from workloads import H, S, T as TG, X
    unitary = [Fragment(wires=[(0, 1)], gates=[(g, 0, -1) for g in gs], qin=[(0, 0)], qout=[(1, 0)],
                        marg=[], slots=[0, 1], clifford=TG not in gs)
               for gs in ([H], [H, TG], [S, H, TG, X], [TG, H, S])]
    for f in _fragments_with_inputs() + unitary:
        T = exact_tensor(f)
        assert is_physical(f, T, tol=1e-10)
        J = choi_blocks(f, T)
        # per-input trace preservation: partial trace over the output slots
        kinds = slot_is_input(f)
        d = len(kinds)
        Jsum = J.sum(axis=0).reshape([2] * (2 * d))
        for j in reversed(range(d)):          # slot j = Kronecker factor j
            if not kinds[j]:
                Jsum = np.trace(Jsum, axis1=j, axis2=j + Jsum.ndim // 2)
        din = 1 << sum(kinds)
        assert np.abs(Jsum.reshape(din, din) - np.eye(din)).max() < 1e-10
    for f in unitary:
        w = np.linalg.eigvalsh(choi_blocks(f, exact_tensor(f), transpose_inputs=False))
        assert w.min() < -0.9


def test_choi_round_trip():
    rng = np.random.default_rng(1)
    f = _fragments_with_inputs()[1]
    T = rng.normal(size=(1 << len(f.marg), 4 ** len(f.slots)))
    assert np.abs(tensor_from_choi(f, choi_blocks(f, T)) - T).max() < 1e-12


def test_simplex_projection_worked_case():
    x, theta = project_simplex([0.6, 0.5, -0.1], 1.0)
    assert np.allclose(x, [0.55, 0.45, 0.0], atol=1e-15) and abs(theta - 0.05) < 1e-15
    x, theta = project_simplex([3.0, 1.0, 0.0, -2.0], 2.0)     # only the largest survives
    assert np.allclose(x, [2.0, 0, 0, 0], atol=1e-15) and abs(theta - 1.0) < 1e-15
    x, _ = project_simplex([0.2, 0.3, 0.5], 1.0)                 # already feasible
    assert np.allclose(x, [0.2, 0.3, 0.5], atol=1e-15)


@pytest.mark.parametrize("seed", range(4))
def test_simplex_projection_is_the_nearest_feasible_point(seed):
    """Feasible, of the form max(lam - theta, 0), and no farther from lam than
    any of many random feasible points (brute force)."""
    rng = np.random.default_rng(seed)
    lam = rng.normal(size=12) * 0.5 + 0.1
    x, theta = project_simplex(lam, 2.0)
    assert x.min() >= 0 and abs(x.sum() - 2.0) < 1e-12
    assert np.allclose(x, np.maximum(lam - theta, 0))
    d0 = np.linalg.norm(lam - x)
    Y = rng.dirichlet(np.full(12, 0.3), size=20000) * 2.0
    assert (np.linalg.norm(Y - lam, axis=1) >= d0 - 1e-12).all()


def _sampled(w, shots, seed):
    return evaluate(w.circuit, w.cuts, w.marginal, (), mode="sampled", shots=shots,
                    seed_lo=seed, seed_hi=0x77)


def test_correction_is_the_nearest_physical_model():
    """On noisy (few-shot) fragment tensors: the corrected model is physical,
    and first-order optimal -- Re Tr[(J' - J)(Y - J')] >= 0 for physical Y
    (random block-diagonal PSD operators of the right total trace, and the
    exact model), which by convexity makes it the nearest physical model."""
    c, cuts = tree_circuit([0, 1], 10, 2, seed=3)
    w = Workload("t", c, cuts, [0, 2, c.n_qubits - 1], [], 24, 1)
    res = _sampled(w, 24, 0x51)
    ex = evaluate(c, cuts, w.marginal, (), mode="exact")
    rng = np.random.default_rng(9)
    corrected = 0
    for f, T, Te in zip(res.fragments, res.tensors, ex.tensors):
        Tc, info = ml_correct(f, T)
        assert is_physical(f, Tc, tol=1e-9)
        J, Jc = choi_blocks(f, T), choi_blocks(f, Tc)
        if info["min_eig"] < -1e-9:
            corrected += 1
        else:
            assert np.abs(Tc - T).max() < 1e-9          # already physical: unchanged
        G = Jc - J
        cands = [choi_blocks(f, Te)]
        nb, D = J.shape[0], J.shape[1]
        for _ in range(30):
            A = rng.normal(size=(nb, D, D)) + 1j * rng.normal(size=(nb, D, D))
            Y = A @ np.conj(np.transpose(A, (0, 2, 1)))
            Y *= 2 ** len(f.qin) / np.trace(Y, axis1=1, axis2=2).real.sum()
            cands.append(Y)
        for Y in cands:
            assert np.einsum("oab,oba->", G, Y - Jc).real >= -1e-9
    assert corrected > 0


def test_exact_models_are_fixed_points():
    c, cuts = tree_circuit([0, 0], 10, 1, seed=5)
    ex = evaluate(c, cuts, [0, 1, c.n_qubits - 1], (), mode="exact")
    for f, T in zip(ex.fragments, ex.tensors):
        Tc, _ = ml_correct(f, T)
        assert np.abs(Tc - T).max() < 1e-10


def test_correction_removes_negative_quasi_probabilities():
    """A star sampled with few shots: the raw contraction has negative
    entries; with every fragment corrected the contraction is a composition
    of completely positive maps, so no entry is negative, and it lies closer
    to the uncut statevector's marginal (Hellinger fidelity, fixed seeds)."""
    w = small_star()
    bf, _ = brute_force(w.circuit, w.marginal)
    raw_neg = 0
    fid_raw, fid_ml = [], []
    for seed in range(4):
        res = _sampled(w, 64, 0x100 + seed)
        k = res.meta["k"]
        Tc = [ml_correct(f, T)[0] for f, T in zip(res.fragments, res.tensors)]
        p_ml = recombine(res.fragments, Tc, k, len(w.marginal))
        raw_neg += (res.marginal < -1e-12).any()
        assert p_ml.min() >= -1e-12
        fid_raw.append(np.sum(np.sqrt(np.clip(res.marginal, 0, None) * bf)) ** 2)
        fid_ml.append(np.sum(np.sqrt(p_ml * bf)) ** 2)
    assert raw_neg > 0
    assert np.mean(fid_ml) > np.mean(fid_raw)


def test_cut_free_fragment_is_the_simplex_projection():
    """A fragment without cut slots has 1 x 1 Choi blocks (its marginal
    distribution): the correction is the plain Euclidean projection of that
    vector onto the probability simplex (total 2^0 = 1)."""
    f = Fragment(wires=[(0, 0), (1, 0)], gates=[], qin=[], qout=[], marg=[(0, 0), (1, 1)], slots=[])
    T = np.array([[0.6], [0.5], [-0.1], [0.0]])
    Tc, info = ml_correct(f, T)
    want, theta = project_simplex(T[:, 0], 1.0)
    assert np.abs(Tc[:, 0] - want).max() < 1e-15 and abs(info["theta"] - theta) < 1e-15
    assert np.allclose(Tc[:, 0], [0.55, 0.45, 0.0, 0.0])
