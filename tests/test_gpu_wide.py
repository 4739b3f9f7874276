"""Clifford fragments wider than a per-variant tableau fits in shared memory.

The default path evolves each Clifford fragment's body once, keeps it in
global memory (one 64-row word of every column per CTA while it evolves) and
derives every variant's outcome space from it, so it is not bound by the
640 wires a whole tableau in shared memory allows.  Here a 1002-wire body
(the "thousands of qubits" regime of Sec. III-A, for stabilizer tableaus):
outcome spaces of sampled variants bit-exact against the oracle's tableau,
and with every T replaced by S (a Clifford circuit) the exact and stitched
marginals equal one uncut tableau's closed form.  Keeping per-variant
tableaus of such a fragment is refused.
"""
import numpy as np
import pytest

from paper_2303_10788_gb300 import ccs
from workloads import Region, Workload, brickwork_star, t_to_s
from oracle.pipeline import evaluate_workload, uncut_clifford

pytestmark = pytest.mark.gpu


def wide_star():
    regs = [Region([0], 1, 4, 10, [0, 1], 2), Region([501], 502, 5, 11, [501, 502], 2)]
    c, cuts = brickwork_star(1002, 12, regs, seed=11)
    marg = [0, 501, 3, 90, 200, 333, 499, 600, 700, 808, 900, 1001]
    return Workload("wide1002", c, cuts, marg, [], 1024, 11)


@pytest.fixture(scope="module")
def ctx():
    return ccs.ccs_create(0)


def test_wide_body_outcome_spaces(ctx):
    w = wide_star()
    plan = ccs.ccs_build_fragments(ctx, [w])
    nf, nc = ccs.ccs_plan_counts(ctx, plan, 0)
    infos = [ccs.ccs_fragment_info_get(ctx, plan, 0, f) for f in range(nf)]
    body = max(range(nf), key=lambda f: infos[f]["n_wires"])
    assert infos[body]["n_wires"] == 1002 and infos[body]["clifford"] and nc == 4
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=w.shots, seed_lo=5, seed_hi=6)
    marg, _ = ccs.ccs_recombine(ctx, plan, res)
    assert np.isfinite(marg).all()
    vs = [0, 77, infos[body]["n_variants"] - 1]
    orc = evaluate_workload(w, mode="sampled", seed_lo=5, seed_hi=6, variants_only={body: vs},
                            keep_tableaus=False)
    for i, v in enumerate(vs):
        ov = orc.variants[body][i]
        off, B, _ = ccs.ccs_get_outcome_space(ctx, res, 0, body, v)
        assert (off, B) == (ov.off, list(ov.basis)), v
    with pytest.raises(ccs.CCSError) as e:
        ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=64, keep_tableaus=True)
    assert "UNSUPPORTED" in str(e.value)


def test_wide_body_t_to_s_exact_and_stitched(ctx):
    w = wide_star()
    c = t_to_s(w.circuit)
    ws = Workload("wide_s", c, w.cuts, w.marginal, [], w.shots, w.seed)
    plan = ccs.ccs_build_fragments(ctx, [ws])
    cf, _ = uncut_clifford(c, w.marginal)
    for mode in (ccs.CCS_EXACT, ccs.CCS_STITCH):
        res = ccs.ccs_eval_variants(ctx, plan, mode=mode)
        m, _ = ccs.ccs_recombine(ctx, plan, res)
        assert np.abs(m - cf).max() < 1e-5, mode
