"""Config 4: many independent circuits (50-300 qubits, 1-3 regions) in one
plan, evaluated by the same persistent launches (needs a GPU).

Exact mode with every T replaced by S must reproduce each circuit's
closed-form marginal; in sampled mode a few variants of a few circuits are
compared bit-exactly with the oracle (the problem index is the Philox
counter's last word).
"""
import numpy as np
import pytest

from paper_2303_10788_gb300 import ccs
from workloads import Workload, config4, t_to_s
from oracle.pipeline import evaluate_workload, uncut_clifford

pytestmark = pytest.mark.gpu
SEED = (0x1234, 0x5678)


@pytest.fixture(scope="module")
def ctx():
    return ccs.ccs_create(0)


def test_config4_batch_t_to_s_exact(ctx):
    ws = []
    for w in config4(256)[:48]:
        ws.append(Workload(w.name, t_to_s(w.circuit), w.cuts, w.marginal, [], w.shots, w.seed))
    plan = ccs.ccs_build_fragments(ctx, ws)
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_EXACT, use_graph=True)
    marg, _ = ccs.ccs_recombine(ctx, plan, res)
    off = 0
    for w in ws:
        nm = 1 << len(w.marginal)
        cf, _ = uncut_clifford(w.circuit, w.marginal)
        assert np.abs(marg[off:off + nm] - cf).max() < 1e-5, w.name
        off += nm


def test_config4_batch_sampled_variants(ctx):
    ws = config4(256)[:24]
    plan = ccs.ccs_build_fragments(ctx, ws)
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=ws[0].shots, seed_lo=SEED[0],
                                seed_hi=SEED[1], keep_tableaus=True)
    marg, _ = ccs.ccs_recombine(ctx, plan, res)
    assert np.all(np.isfinite(marg))
    rng = np.random.default_rng(0)
    for pi in (0, 7, 23):
        nf, _ = ccs.ccs_plan_counts(ctx, plan, pi)
        only = {}
        for f in range(nf):
            info = ccs.ccs_fragment_info_get(ctx, plan, pi, f)
            nv = info["n_variants"]
            only[f] = sorted(set([0, nv - 1] + [int(x) for x in rng.choice(nv, size=min(2, nv), replace=False)]))
        orc = evaluate_workload(ws[pi], mode="sampled", seed_lo=SEED[0], seed_hi=SEED[1], circuit_id=pi,
                                variants_only=only)
        for f, lst in only.items():
            info = ccs.ccs_fragment_info_get(ctx, plan, pi, f)
            for i, v in enumerate(lst):
                ov = orc.variants[f][i]
                if info["clifford"]:
                    assert np.array_equal(ccs.ccs_get_tableau(ctx, res, pi, f, v), ov.tableau), (pi, f, v)
                    o, B, _ = ccs.ccs_get_outcome_space(ctx, res, pi, f, v)
                    assert (o, B) == (ov.off, list(ov.basis)), (pi, f, v)
                    cnt = ccs.ccs_get_counts(ctx, res, pi, f, v).astype(np.int64)
                    assert np.array_equal(cnt, ov.counts), (pi, f, v)
                else:
                    assert np.abs(ccs.ccs_get_dist(ctx, res, pi, f, v) - ov.dist).max() < 2e-6
