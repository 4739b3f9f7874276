"""Config 3 at full size: 500-qubit Clifford body (1000 x 1001-bit tableau in
shared memory), 20736 body variants, 2^14 shots each, 8 cuts (4^8 cut
terms), 16-qubit marginal (needs a GPU).

The oracle cannot evaluate all 20736 variants in test time, so: sampled
variants are compared bit-exactly one by one, and the whole path is pinned at
full size by the T->S property (exact mode must reproduce one uncut
tableau's closed-form marginal), in FP32 (gated at 1e-5) and BF16 (stated).
"""
import numpy as np
import pytest

from paper_2303_10788_gb300 import ccs
from workloads import Workload, config3, t_to_s
from oracle.pipeline import evaluate_workload, uncut_clifford

pytestmark = pytest.mark.gpu
SEED = (0x1234, 0x5678)


@pytest.fixture(scope="module")
def ctx():
    return ccs.ccs_create(0)


def test_config3_sampled_variants_bit_exact(ctx):
    w = config3()
    plan = ccs.ccs_build_fragments(ctx, [w])
    nf, nc = ccs.ccs_plan_counts(ctx, plan, 0)
    infos = [ccs.ccs_fragment_info_get(ctx, plan, 0, f) for f in range(nf)]
    body = max(range(nf), key=lambda f: infos[f]["n_wires"])
    assert infos[body]["n_wires"] == 500 and infos[body]["n_variants"] == 20736 and nc == 8
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=w.shots, seed_lo=SEED[0],
                                seed_hi=SEED[1], keep_tableaus=True)
    marg, _ = ccs.ccs_recombine(ctx, plan, res)
    rng = np.random.default_rng(3)
    vs = sorted(int(v) for v in rng.choice(20736, size=5, replace=False)) + [0, 20735]
    only = {body: vs}
    for f in range(nf):
        if f != body:
            only[f] = list(range(12))
    orc = evaluate_workload(w, mode="sampled", seed_lo=SEED[0], seed_hi=SEED[1], variants_only=only)
    for f, lst in only.items():
        for i, v in enumerate(lst):
            ov = orc.variants[f][i]
            if infos[f]["clifford"]:
                assert np.array_equal(ccs.ccs_get_tableau(ctx, res, 0, f, v), ov.tableau), (f, v)
                off, B, _ = ccs.ccs_get_outcome_space(ctx, res, 0, f, v)
                assert (off, B) == (ov.off, list(ov.basis)), (f, v)
                assert np.array_equal(ccs.ccs_get_counts(ctx, res, 0, f, v).astype(np.int64), ov.counts), (f, v)
            else:
                assert np.abs(ccs.ccs_get_dist(ctx, res, 0, f, v) - ov.dist).max() < 2e-6
    # sampled-mode quasi-probabilities: normalised up to shot noise
    assert abs(marg.sum() - 1.0) < 0.05


def test_config3_t_to_s_exact_full_size(ctx):
    w = config3()
    c = t_to_s(w.circuit)
    ws = Workload("c3s", c, w.cuts, w.marginal, [], w.shots, w.seed)
    plan = ccs.ccs_build_fragments(ctx, [ws])
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_EXACT)
    m32, _ = ccs.ccs_recombine(ctx, plan, res, precision=ccs.CCS_FP32)
    m16, _ = ccs.ccs_recombine(ctx, plan, res, precision=ccs.CCS_BF16)
    cf, _ = uncut_clifford(c, w.marginal)
    e32, e16 = np.abs(m32 - cf).max(), np.abs(m16 - cf).max()
    print(f"config3 T->S exact: max|err| fp32={e32:.2e} bf16={e16:.2e} (max p={cf.max():.2e})")
    assert e32 < 1e-5
    assert e16 < 1e-3


def test_config3_bf16_tensor_cores_match_cuda_cores(ctx):
    """The tcgen05 BF16 GEMM and the CUDA-core BF16 path multiply the same
    bf16-rounded operands; only the FP32 accumulation order differs."""
    w = config3()
    plan = ccs.ccs_build_fragments(ctx, [w])
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=w.shots, seed_lo=SEED[0], seed_hi=SEED[1])
    m_tc, _ = ccs.ccs_recombine(ctx, plan, res, precision=ccs.CCS_BF16)
    m_cc, _ = ccs.ccs_recombine(ctx, plan, res, precision=ccs.CCS_BF16, tensor_cores=False)
    m32, _ = ccs.ccs_recombine(ctx, plan, res, precision=ccs.CCS_FP32)
    d = np.abs(m_tc - m_cc).max()
    print(f"config3 sampled: |tc - cuda-core bf16| = {d:.2e}, |bf16 - fp32| = {np.abs(m_tc - m32).max():.2e}, "
          f"max|p| = {np.abs(m32).max():.2e}")
    assert d < 1e-6 * max(1.0, np.abs(m32).max() * 1e3)
