"""The byte-counter hub sampler against the 16-bit one (needs a GPU).

Both count the same Philox shots, so the hubs' dense counts, the hub
operands and the recombined marginals must agree bit for bit.  The
workloads cover both paths of the byte kernel: config 2's hub (rank 6,
10^4 shots > 64 * 2^6: recounted with 16-bit counters in two passes over
the output halves) and config 3 / config 4 hubs (full rank: byte counters).
"""
import numpy as np
import pytest

from paper_2303_10788_gb300 import ccs
from workloads import config2, config3, config4

pytestmark = pytest.mark.gpu
SEED = (0x1234, 0x5678)


@pytest.fixture(scope="module")
def ctx():
    return ccs.ccs_create(0)


@pytest.mark.parametrize("make", [lambda: [config2()], lambda: config4(64)[:16], lambda: [config3()]],
                         ids=["config2", "config4x16", "config3"])
def test_byte_sampler_equals_16bit(ctx, make):
    ws = make()
    plan = ccs.ccs_build_fragments(ctx, ws)
    kw = dict(mode=ccs.CCS_SAMPLED, shots=ws[0].shots, seed_lo=SEED[0], seed_hi=SEED[1], keep_tableaus=True)
    r16 = ccs.ccs_eval_variants(ctx, plan, hub_sampler=1, **kw)
    r8 = ccs.ccs_eval_variants(ctx, plan, hub_sampler=2, **kw)
    r8w = ccs.ccs_eval_variants(ctx, plan, hub_sampler=3, **kw)      # byte counters, 512-thread CTAs
    assert ccs.ccs_get_tuning(ctx, r8)[3] == -256 and ccs.ccs_get_tuning(ctx, r8w)[3] == -512
    assert ccs.ccs_get_tuning(ctx, r16)[3] > 0
    m16, z16 = ccs.ccs_recombine(ctx, plan, r16)
    m8, z8 = ccs.ccs_recombine(ctx, plan, r8)
    m8w, z8w = ccs.ccs_recombine(ctx, plan, r8w)
    assert np.array_equal(m16, m8) and np.array_equal(z16, z8)
    assert np.array_equal(m8w, m8) and np.array_equal(z8w, z8)
    for f in range(ccs.ccs_plan_counts(ctx, plan, 0)[0]):
        info = ccs.ccs_fragment_info_get(ctx, plan, 0, f)
        if info["clifford"] and info["n_slots"] == ccs.ccs_plan_counts(ctx, plan, 0)[1]:
            for v in range(0, info["n_variants"], max(1, info["n_variants"] // 7)):
                assert np.array_equal(ccs.ccs_get_counts(ctx, r8w, 0, f, v), ccs.ccs_get_counts(ctx, r8, 0, f, v))
    rng = np.random.default_rng(0)
    checked = 0
    for pi in range(len(ws)):
        nf, k = ccs.ccs_plan_counts(ctx, plan, pi)
        for f in range(nf):
            info = ccs.ccs_fragment_info_get(ctx, plan, pi, f)
            if not info["clifford"] or info["n_slots"] != k:
                continue
            nv = info["n_variants"]
            for v in sorted(set([0, nv - 1] + [int(x) for x in rng.choice(nv, size=min(4, nv), replace=False)])):
                assert np.array_equal(ccs.ccs_get_counts(ctx, r16, pi, f, v), ccs.ccs_get_counts(ctx, r8, pi, f, v))
                checked += 1
            assert np.array_equal(ccs.ccs_get_operand(ctx, r16, pi, f), ccs.ccs_get_operand(ctx, r8, pi, f))
    assert checked >= 2
