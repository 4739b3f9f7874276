"""The largest workloads on the benchmark's own path against stored oracle results.

Config 3 (500-qubit Clifford body, 20736 variants, 2^14 shots each, 8 cuts,
4^8 cut terms, 16-qubit marginal, 16 T gates) and the first config-4 circuits
(evaluated inside the full 256-circuit plan), run exactly as bench.py times
them: sampled mode with the benchmark's seed, shared bodies and the
outcome-space screen (no tableaus kept), the hub sampler folding its shots
straight into the contraction operand, CUDA graphs, autotuned launch shapes.
The expected values were written by tests/golden/make_golden.py, which calls
only the oracle (FP64): the recombined marginal (Sec. V-C) and every Clifford
variant's canonical outcome space (off, reduced basis).

Bars: outcome spaces bit-exact; FP32 marginal within 1e-5 absolute (the
spec bound); the BF16 tensor-core contraction's error against the FP64
oracle is printed and held under 2e-4 (its operands carry 8 significant bits).
The same config-4 run with every Clifford fragment's model corrected by
maximum likelihood (Sec. V-C) before the contraction is held to 1e-5 against
the oracle's corrected contraction, and no entry of any of the 256 corrected
marginals is negative.
"""
import os

import numpy as np
import pytest

from paper_2303_10788_gb300 import ccs
from workloads import config3, config4

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
GOLD3 = os.path.join(HERE, "golden", "config3_sampled.npz")
GOLD4 = os.path.join(HERE, "golden", "config4_sampled.npz")
GOLDML = os.path.join(HERE, "golden", "ml_marginals.npz")


@pytest.fixture(scope="module")
def ctx():
    return ccs.ccs_create(0)


def _bench_eval(ctx, ws, seed):
    plan = ccs.ccs_build_fragments(ctx, ws)
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=ws[0].shots, seed_lo=int(seed[0]),
                                seed_hi=int(seed[1]), use_graph=True, autotune=True)
    return plan, res


def _check_spaces(ctx, res, problem, rows):
    """rows: (fragment, variant, rank, off, basis...) per Clifford variant."""
    bad = 0
    for r in rows:
        f, v, rank, off = int(r[0]), int(r[1]), int(r[2]), int(r[3])
        o, B, rk = ccs.ccs_get_outcome_space(ctx, res, problem, f, v)
        if (rk, o, B) != (rank, off, [int(b) for b in r[4:4 + rank]]):
            bad += 1
    return bad


def test_config3_default_path_matches_oracle(ctx):
    g = np.load(GOLD3)
    w = config3()
    plan, res = _bench_eval(ctx, [w], g["seed"])
    # every body variant's outcome space, from the screen (no tableau formed)
    body, sp = int(g["body"]), g["spaces"]
    rows = np.concatenate([np.full((len(sp), 1), body, np.uint32),
                           np.arange(len(sp), dtype=np.uint32)[:, None], sp], axis=1)
    assert _check_spaces(ctx, res, 0, rows) == 0
    gold = g["marginal"]
    m32, _ = ccs.ccs_recombine(ctx, plan, res, precision=ccs.CCS_FP32, use_graph=True)
    m16, _ = ccs.ccs_recombine(ctx, plan, res, precision=ccs.CCS_BF16, use_graph=True)
    e32, e16 = np.abs(m32 - gold).max(), np.abs(m16 - gold).max()
    print(f"config3 sampled vs FP64 oracle: max|err| fp32 {e32:.2e}, bf16 (tcgen05) {e16:.2e}, "
          f"L1 bf16 {np.abs(m16 - gold).sum():.2e}, max|p| {np.abs(gold).max():.2e}")
    assert e32 < 1e-5
    assert e16 < 2e-4
    # a replay of the evaluation graph reproduces the marginal bit for bit
    ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=w.shots, seed_lo=int(g["seed"][0]),
                          seed_hi=int(g["seed"][1]), use_graph=True, res=res)
    m32b, _ = ccs.ccs_recombine(ctx, plan, res, precision=ccs.CCS_FP32, use_graph=True)
    assert np.array_equal(m32, m32b)


def test_config4_default_path_matches_oracle(ctx):
    g = np.load(GOLD4)
    ws = config4(256)
    plan, res = _bench_eval(ctx, ws, g["seed"])
    m32, _ = ccs.ccs_recombine(ctx, plan, res, precision=ccs.CCS_FP32, use_graph=True)
    m16, _ = ccs.ccs_recombine(ctx, plan, res, precision=ccs.CCS_BF16, use_graph=True)
    offs = np.concatenate([[0], np.cumsum([1 << len(w.marginal) for w in ws])])
    worst32 = worst16 = 0.0
    for i, ci in enumerate(g["circuits"]):
        ci = int(ci)
        assert _check_spaces(ctx, res, ci, g[f"spaces_{ci}"]) == 0, ci
        gold = g["marginals"][i]
        worst32 = max(worst32, np.abs(m32[offs[ci]:offs[ci + 1]] - gold).max())
        worst16 = max(worst16, np.abs(m16[offs[ci]:offs[ci + 1]] - gold).max())
    print(f"config4 circuits {list(g['circuits'])} vs FP64 oracle: max|err| fp32 {worst32:.2e}, bf16 {worst16:.2e}")
    assert worst32 < 1e-5
    assert worst16 < 2e-4


def test_config4_ml_correction_matches_oracle(ctx):
    g = np.load(GOLDML)
    ws = config4(256)
    plan, res = _bench_eval(ctx, ws, g["seed"])
    ccs.ccs_ml_correct(ctx, plan, res, ccs.CCS_ML_SAMPLED)
    m, _ = ccs.ccs_recombine(ctx, plan, res, precision=ccs.CCS_FP32, use_graph=True)
    offs = np.concatenate([[0], np.cumsum([1 << len(w.marginal) for w in ws])])
    worst = 0.0
    for i, ci in enumerate(g["config4_circuits"]):
        ci = int(ci)
        worst = max(worst, np.abs(m[offs[ci]:offs[ci + 1]] - g["config4"][i]).max())
    print(f"config4 ML-corrected vs FP64 oracle: max|err| {worst:.2e}; min entry over 256 circuits {m.min():.2e}")
    assert worst < 1e-5
    assert m.min() > -1e-5
