"""The paper's benchmark shapes and Z^a gates on the GPU, against the oracle.

HWEA (5 rounds, one injected T, up to the paper's 300 qubits) and SK-model
MaxCut QAOA (one round, all-to-all, up to the paper's 26 qubits), Sec. VI-B;
Z^a rotations with 2a not an integer as the non-Clifford gates (Sec. VIII).
No cut set is given: the library's search chooses it, and the oracle is run
on the cuts the plan reports.  Bit-exact tableaus, outcome spaces and shot
counts; distributions within 2e-6; recombined results within 1e-5; in exact
mode also the uncut statevector where it fits (<= 16 qubits).
"""
import numpy as np
import pytest

from paper_2303_10788_gb300 import ccs
from workloads import hwea, sk_qaoa
from oracle.pipeline import evaluate, brute_force
from test_gpu_parity import check_variants, SEED, TOL_MARG

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return ccs.ccs_create(0)


CASES = {
    "hwea16": hwea(16, rounds=5, n_t=1, n_z=8),
    "hwea300": hwea(300, rounds=5, n_t=1, n_z=8),
    "hwea20_zpow": hwea(20, rounds=5, n_t=3, n_z=8, zpow=True),
    "skqaoa12_zpow": sk_qaoa(12, n_t=2, n_z=8, zpow=True),
    "skqaoa26": sk_qaoa(26, n_t=1, n_z=8),
}


@pytest.mark.parametrize("mode", [ccs.CCS_EXACT, ccs.CCS_SAMPLED])
@pytest.mark.parametrize("name", list(CASES))
def test_paper_workload(ctx, name, mode):
    w = CASES[name]
    plan = ccs.ccs_build_fragments(ctx, [w])
    cuts = ccs.ccs_plan_cuts(ctx, plan, 0)
    res = ccs.ccs_eval_variants(ctx, plan, mode=mode, shots=w.shots, seed_lo=SEED[0], seed_hi=SEED[1],
                                keep_tableaus=True)
    marg, zexp = ccs.ccs_recombine(ctx, plan, res)
    orc = evaluate(w.circuit, cuts, w.marginal, w.zstrings,
                   mode="exact" if mode == ccs.CCS_EXACT else "sampled", shots=w.shots,
                   seed_lo=SEED[0], seed_hi=SEED[1])
    check_variants(ctx, res, orc, mode)
    assert np.abs(marg - orc.marginal).max() < TOL_MARG
    assert np.abs(zexp - orc.zexp).max() < TOL_MARG
    if mode == ccs.CCS_EXACT and w.circuit.n_qubits <= 16:
        bf, bz = brute_force(w.circuit, w.marginal, w.zstrings)
        assert np.abs(marg - bf).max() < TOL_MARG
        assert np.abs(zexp - bz).max() < TOL_MARG


def test_zpow_statevector_precision(ctx):
    """Non-Clifford Z^a at exponents far from 0 and beyond one period: the
    library reduces a mod 2 before forming e^{i pi a}; the fragment
    distributions still match the oracle's complex128 statevector."""
    w = hwea(12, rounds=3, n_t=0, n_z=4)
    rng = np.random.default_rng(5)
    for a in (1e3 + 0.3, -77.71, 2.0 ** 40 + 0.25, 0.001):
        w.circuit.gates.insert(int(rng.integers(len(w.circuit.gates))), (10, int(rng.integers(12)), -1, a))
    plan = ccs.ccs_build_fragments(ctx, [w])
    cuts = ccs.ccs_plan_cuts(ctx, plan, 0)
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_EXACT, keep_tableaus=True)
    marg, zexp = ccs.ccs_recombine(ctx, plan, res)
    orc = evaluate(w.circuit, cuts, w.marginal, w.zstrings, mode="exact")
    check_variants(ctx, res, orc, ccs.CCS_EXACT)
    bf, bz = brute_force(w.circuit, w.marginal, w.zstrings)
    assert np.abs(marg - bf).max() < TOL_MARG
    assert np.abs(zexp - bz).max() < TOL_MARG
