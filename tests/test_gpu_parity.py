"""GPU path vs the oracle through the C ABI (needs a GPU).

Bit-exact: final tableaus, canonical outcome spaces (off, basis) and Philox
shot counts.  Floating point: non-Clifford variant distributions within
2e-6, recombined marginals and <Z_S> within 1e-5 absolute (FP32 operands,
FP32 accumulation over 64-term chunks, FP64 across chunks).
"""
import numpy as np
import pytest

from paper_2303_10788_gb300 import ccs
from workloads import (Circuit, Region, Workload, brickwork_star, config1, config2, small_star,
                       random_clifford_circuit, zstrings_for, t_to_s, CX, H, S, T)
from oracle.pipeline import evaluate, evaluate_workload, uncut_clifford

pytestmark = pytest.mark.gpu

SEED = (0x1234, 0x5678)
TOL_MARG = 1e-5


@pytest.fixture(scope="module")
def ctx():
    return ccs.ccs_create(0)


def gpu_run(ctx, ws, mode, keep=True, shots=None, precision=ccs.CCS_FP32, use_graph=False):
    plan = ccs.ccs_build_fragments(ctx, ws)
    res = ccs.ccs_eval_variants(ctx, plan, mode=mode, shots=shots or ws[0].shots, seed_lo=SEED[0],
                                seed_hi=SEED[1], keep_tableaus=keep, use_graph=use_graph)
    marg, zexp = ccs.ccs_recombine(ctx, plan, res, precision=precision)
    return plan, res, marg, zexp


def check_variants(ctx, res, orc, mode, problem=0, only=None):
    for fi, f in enumerate(orc.fragments):
        vs = range(f.n_variants) if only is None else only.get(fi, [])
        for idx, v in enumerate(vs):
            ov = orc.variants[fi][v if only is None else idx]
            if f.clifford:
                tab = ccs.ccs_get_tableau(ctx, res, problem, fi, v)
                assert np.array_equal(tab, ov.tableau), (fi, v, "tableau")
                off, B, rank = ccs.ccs_get_outcome_space(ctx, res, problem, fi, v)
                assert (off, B) == (ov.off, list(ov.basis)), (fi, v, "space")
                if mode == ccs.CCS_SAMPLED:
                    cnt = ccs.ccs_get_counts(ctx, res, problem, fi, v)
                    assert np.array_equal(cnt.astype(np.int64), ov.counts), (fi, v, "counts")
                else:
                    d = ccs.ccs_get_dist(ctx, res, problem, fi, v)
                    assert np.array_equal(d.astype(np.float64), ov.dist), (fi, v, "exact dist")
            else:
                d = ccs.ccs_get_dist(ctx, res, problem, fi, v)
                assert np.abs(d - ov.dist).max() < 2e-6, (fi, v, "statevector")


SMALL = [
    small_star(),
    small_star(n=9, depth=7, region_full=(0, 1, 2), boundary=3, window=(2, 5), n_t=2, seed=5),
    small_star(n=6, depth=5, region_full=(0,), boundary=1, window=(1, 3), n_t=1, seed=9),
    small_star(n=12, depth=9, region_full=(0, 1, 2, 3), boundary=4, window=(2, 6), n_t=3, seed=3),
]


@pytest.mark.parametrize("mode", [ccs.CCS_EXACT, ccs.CCS_SAMPLED])
@pytest.mark.parametrize("wi", range(len(SMALL)))
def test_small_stars(ctx, wi, mode):
    w = SMALL[wi]
    orc = evaluate_workload(w, mode="exact" if mode == ccs.CCS_EXACT else "sampled",
                            seed_lo=SEED[0], seed_hi=SEED[1])
    plan, res, marg, zexp = gpu_run(ctx, [w], mode)
    check_variants(ctx, res, orc, mode)
    for fi, T_ in enumerate(orc.tensors):
        assert np.abs(ccs.ccs_get_tensor(ctx, res, 0, fi) - T_).max() < 1e-5
    assert np.abs(marg - orc.marginal).max() < TOL_MARG
    assert np.abs(zexp - orc.zexp).max() < TOL_MARG


@pytest.mark.parametrize("mode", [ccs.CCS_EXACT, ccs.CCS_SAMPLED])
def test_config1(ctx, mode):
    w = config1()
    orc = evaluate_workload(w, mode="exact" if mode == ccs.CCS_EXACT else "sampled",
                            seed_lo=SEED[0], seed_hi=SEED[1])
    plan, res, marg, zexp = gpu_run(ctx, [w], mode)
    check_variants(ctx, res, orc, mode)
    assert np.abs(marg - orc.marginal).max() < TOL_MARG
    assert np.abs(zexp - orc.zexp).max() < TOL_MARG


@pytest.mark.parametrize("n_body", [62, 63, 64, 65, 127, 128, 129])
def test_word_boundaries(ctx, n_body):
    """Body widths around multiples of 64 rows (ragged last word)."""
    # region = qubit 0 plus a window of qubit 1; qubit 1 leaves two body
    # wires, so the body has exactly n_body wires
    reg = Region([0], 1, 2, 5, [0, 1], 2)
    c, cuts = brickwork_star(n_body, 7, [reg], seed=n_body)
    rng = np.random.default_rng(n_body)
    w = Workload(f"wb{n_body}", c, cuts, [0, 1, 5, n_body - 1], zstrings_for(n_body, 6, rng, 5),
                 3000, 7, [reg])
    orc = evaluate_workload(w, mode="sampled", seed_lo=SEED[0], seed_hi=SEED[1])
    plan, res, marg, zexp = gpu_run(ctx, [w], ccs.CCS_SAMPLED)
    check_variants(ctx, res, orc, ccs.CCS_SAMPLED)
    assert np.abs(marg - orc.marginal).max() < TOL_MARG
    assert np.abs(zexp - orc.zexp).max() < TOL_MARG


def test_no_cuts_clifford_and_nc(ctx):
    """Degenerate plans: one Clifford fragment, one non-Clifford fragment, and
    a circuit with an idle qubit (a cut-free extra fragment)."""
    c1 = random_clifford_circuit(20, 300, seed=4)
    c2 = random_clifford_circuit(6, 60, seed=5, t_count=3)
    c3 = random_clifford_circuit(5, 40, seed=6)
    c3.n_qubits = 6                                      # qubit 5 never touched
    ws = [Workload("c", c1, [], [0, 3, 19], [[0, 1], [5]], 2048, 1),
          Workload("nc", c2, [], [0, 2, 5], [[1, 2]], 2048, 2),
          Workload("idle", c3, [], [0, 5], [[5], [0, 5]], 2048, 3)]
    for mode in (ccs.CCS_EXACT, ccs.CCS_SAMPLED):
        plan, res, marg, zexp = gpu_run(ctx, ws, mode)
        off_m, off_z = 0, 0
        for i, w in enumerate(ws):
            orc = evaluate_workload(w, mode="exact" if mode == ccs.CCS_EXACT else "sampled",
                                    seed_lo=SEED[0], seed_hi=SEED[1], circuit_id=i)
            check_variants(ctx, res, orc, mode, problem=i)
            nm, nz = 1 << len(w.marginal), len(w.zstrings)
            assert np.abs(marg[off_m:off_m + nm] - orc.marginal).max() < TOL_MARG
            assert np.abs(zexp[off_z:off_z + nz] - orc.zexp).max() < TOL_MARG
            off_m += nm
            off_z += nz


def test_shot_count_edges(ctx):
    """Shot counts that are not multiples of the per-CTA chunk, and 1 shot."""
    w = small_star()
    for shots in (1, 255, 4097, 10001):
        orc = evaluate(w.circuit, w.cuts, w.marginal, w.zstrings, "sampled", shots, *SEED)
        plan, res, marg, zexp = gpu_run(ctx, [w], ccs.CCS_SAMPLED, shots=shots)
        check_variants(ctx, res, orc, ccs.CCS_SAMPLED)
        assert np.abs(marg - orc.marginal).max() < TOL_MARG


def test_config2_full_size(ctx):
    """The bench workload at full size, in the bench's launch configuration
    (CUDA graph): all 144 + 2x12 variants and the recombined results."""
    w = config2()
    orc = evaluate_workload(w, mode="sampled", seed_lo=SEED[0], seed_hi=SEED[1])
    plan, res, marg, zexp = gpu_run(ctx, [w], ccs.CCS_SAMPLED, use_graph=True)
    check_variants(ctx, res, orc, ccs.CCS_SAMPLED)
    assert np.abs(marg - orc.marginal).max() < TOL_MARG
    assert np.abs(zexp - orc.zexp).max() < TOL_MARG
    # a second replay of the captured graph reproduces everything
    res2 = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=w.shots, seed_lo=SEED[0],
                                 seed_hi=SEED[1], keep_tableaus=True, use_graph=True, res=res)
    marg2, zexp2 = ccs.ccs_recombine(ctx, plan, res2)
    assert np.array_equal(marg, marg2) and np.array_equal(zexp, zexp2)


def test_t_to_s_exact_large(ctx):
    """T->S at 100 qubits: exact-mode recombination equals one uncut tableau."""
    w = config2()
    c = t_to_s(w.circuit)
    ws = Workload("c2s", c, w.cuts, w.marginal, w.zstrings, w.shots, w.seed)
    plan, res, marg, zexp = gpu_run(ctx, [ws], ccs.CCS_EXACT, keep=False)
    cf, cz = uncut_clifford(c, w.marginal, w.zstrings)
    assert np.abs(marg - cf).max() < TOL_MARG
    assert np.abs(zexp - cz).max() < TOL_MARG


def test_bf16_error_is_reported(ctx):
    """BF16 operands of the contraction: error stated against the FP64 oracle,
    not gated.  Sampled counts over 10^4 shots are not dyadic, so bf16's
    8-bit mantissa shows."""
    w = config2()
    orc = evaluate_workload(w, mode="sampled", seed_lo=SEED[0], seed_hi=SEED[1])
    plan = ccs.ccs_build_fragments(ctx, [w])
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=w.shots, seed_lo=SEED[0],
                                seed_hi=SEED[1])
    m32, _ = ccs.ccs_recombine(ctx, plan, res, precision=ccs.CCS_FP32)
    m16, _ = ccs.ccs_recombine(ctx, plan, res, precision=ccs.CCS_BF16)
    e32, e16 = np.abs(m32 - orc.marginal).max(), np.abs(m16 - orc.marginal).max()
    assert e32 < TOL_MARG
    assert e16 < 1e-3
    print(f"config2 sampled: max|err| fp32={e32:.2e} bf16={e16:.2e} (max p={orc.marginal.max():.2e})")
