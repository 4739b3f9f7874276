"""Parity at the size limits and in degenerate cases (needs a GPU).

The widest Clifford fragment the tableau kernels hold (640 wires, 10 words
per half column, 205 KB of shared memory), the widest statevector fragment
(12 wires, 4096 amplitudes), an empty marginal, a circuit without gates.
"""
import numpy as np
import pytest

from paper_2303_10788_gb300 import ccs
from workloads import Circuit, Region, Workload, brickwork_star, zstrings_for
from oracle.pipeline import evaluate_workload

pytestmark = pytest.mark.gpu
SEED = (0x1234, 0x5678)


@pytest.fixture(scope="module")
def ctx():
    return ccs.ccs_create(0)


def run(ctx, w, mode):
    plan = ccs.ccs_build_fragments(ctx, [w])
    res = ccs.ccs_eval_variants(ctx, plan, mode=mode, shots=w.shots, seed_lo=SEED[0], seed_hi=SEED[1],
                                keep_tableaus=True)
    marg, zexp = ccs.ccs_recombine(ctx, plan, res)
    return plan, res, marg, zexp


def test_widest_tableau_640(ctx):
    reg = Region([0], 1, 2, 4, [0, 1], 2)
    c, cuts = brickwork_star(640, 6, [reg], seed=640)
    rng = np.random.default_rng(640)
    w = Workload("w640", c, cuts, [0, 1, 100, 639], zstrings_for(640, 3, rng, 4), 2000, 7, [reg])
    plan, res, marg, zexp = run(ctx, w, ccs.CCS_SAMPLED)
    infos = [ccs.ccs_fragment_info_get(ctx, plan, 0, f) for f in range(ccs.ccs_plan_counts(ctx, plan, 0)[0])]
    body = max(range(len(infos)), key=lambda f: infos[f]["n_wires"])
    assert infos[body]["n_wires"] == 640
    only = {body: [0, 5, infos[body]["n_variants"] - 1]}
    for f in range(len(infos)):
        if f != body:
            only[f] = list(range(infos[f]["n_variants"]))
    orc = evaluate_workload(w, mode="sampled", seed_lo=SEED[0], seed_hi=SEED[1], variants_only=only)
    for f, vs in only.items():
        for i, v in enumerate(vs):
            ov = orc.variants[f][i]
            if infos[f]["clifford"]:
                assert np.array_equal(ccs.ccs_get_tableau(ctx, res, 0, f, v), ov.tableau), (f, v)
                off, B, _ = ccs.ccs_get_outcome_space(ctx, res, 0, f, v)
                assert (off, B) == (ov.off, list(ov.basis)), (f, v)
                assert np.array_equal(ccs.ccs_get_counts(ctx, res, 0, f, v).astype(np.int64), ov.counts), (f, v)
            else:
                assert np.abs(ccs.ccs_get_dist(ctx, res, 0, f, v) - ov.dist).max() < 2e-6


def test_widest_statevector_12(ctx):
    # region of 11 full qubits + the boundary window: a 12-wire statevector fragment
    reg = Region(list(range(11)), 11, 2, 5, list(range(11)), 4)
    c, cuts = brickwork_star(24, 7, [reg], seed=12)
    rng = np.random.default_rng(12)
    w = Workload("nc12", c, cuts, [0, 5, 10, 11, 17, 23], zstrings_for(24, 4, rng, 4), 4096, 3, [reg])
    plan, res, marg, zexp = run(ctx, w, ccs.CCS_SAMPLED)
    infos = [ccs.ccs_fragment_info_get(ctx, plan, 0, f) for f in range(ccs.ccs_plan_counts(ctx, plan, 0)[0])]
    assert max(i["n_wires"] for i in infos if not i["clifford"]) == 12
    orc = evaluate_workload(w, mode="sampled", seed_lo=SEED[0], seed_hi=SEED[1])
    for f, info in enumerate(infos):
        if not info["clifford"]:
            for v in range(info["n_variants"]):
                assert np.abs(ccs.ccs_get_dist(ctx, res, 0, f, v) - orc.variants[f][v].dist).max() < 2e-6
    assert np.abs(marg - orc.marginal).max() < 1e-5
    assert np.abs(zexp - orc.zexp).max() < 1e-5


def test_empty_marginal_and_gateless_circuit(ctx):
    reg = Region([0, 1], 2, 2, 5, [0, 1], 2)
    c, cuts = brickwork_star(10, 7, [reg], seed=4)
    rng = np.random.default_rng(4)
    w = Workload("nomarg", c, cuts, [], zstrings_for(10, 5, rng, 3), 2048, 5, [reg])
    for mode, m in ((ccs.CCS_EXACT, "exact"), (ccs.CCS_SAMPLED, "sampled")):
        plan, res, marg, zexp = run(ctx, w, mode)
        orc = evaluate_workload(w, mode=m, seed_lo=SEED[0], seed_hi=SEED[1])
        assert marg.shape == (1,)
        assert np.abs(marg - orc.marginal).max() < 1e-5
        assert np.abs(zexp - orc.zexp).max() < 1e-5
    idle = Workload("idle", Circuit(3), [], [0, 2], [[1]], 64, 6)
    for mode in (ccs.CCS_EXACT, ccs.CCS_SAMPLED):
        plan, res, marg, zexp = run(ctx, idle, mode)
        assert np.array_equal(marg, np.array([1.0, 0.0, 0.0, 0.0]))
        assert np.array_equal(zexp, np.array([1.0]))


def test_thirteen_fragments(ctx):
    """The most fragments one problem may have (13: cuts + 1 for 12 cuts, and
    every gate-disconnected wire is a fragment of its own): seven two-qubit
    blocks and five single wires, the first block carrying a T and cut on
    both wires (two fragments), marginal wires in ten different fragments;
    exact and sampled against the oracle."""
    from workloads import CX, H, S, T
    c = Circuit(19)
    for b in range(7):
        a, d = 2 * b, 2 * b + 1
        c.add(H, a); c.add(CX, a, d); c.add(S, d)
    c.add(T, 0)
    g = len(c.gates)                          # the second CX of the first block: both wires cut before it
    c.add(CX, 0, 1); c.add(H, 1)
    for q in range(14, 19):
        c.add(H, q)
    cuts = [(0, g), (1, g)]
    w = Workload("thirteen", c, cuts, [0, 2, 4, 6, 8, 10, 12, 14, 16, 18], [[1, 3], [0, 18]], 1024, 7)
    plan = ccs.ccs_build_fragments(ctx, [w])
    nf, nc = ccs.ccs_plan_counts(ctx, plan, 0)
    assert nf == 13 and nc == 2, (nf, nc)
    for mode, m in ((ccs.CCS_EXACT, "exact"), (ccs.CCS_SAMPLED, "sampled")):
        _, _, marg, zexp = run(ctx, w, mode)
        orc = evaluate_workload(w, mode=m, seed_lo=SEED[0], seed_hi=SEED[1])
        assert np.abs(marg - orc.marginal).max() < 1e-5
        assert np.abs(zexp - orc.zexp).max() < 1e-5
