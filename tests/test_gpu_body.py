"""Shared fragment body vs whole-circuit simulation per variant (needs a GPU).

With body sharing each Clifford fragment's gate sequence is evolved once and
every variant is derived from it by rewriting its input rows; without it
every variant simulates its whole circuit.  Conjugation is exact, so final
tableaus, outcome spaces and shot counts must agree bit for bit, and both
must agree with the oracle (covered by the parity tests, which run the
default shared-body path).
"""
import numpy as np
import pytest

from paper_2303_10788_gb300 import ccs
from workloads import Workload, config1, config2, config4, small_star, hwea, sk_qaoa
from workloads.circuits import zstrings_for

pytestmark = pytest.mark.gpu
SEED = (0x1234, 0x5678)


@pytest.fixture(scope="module")
def ctx():
    return ccs.ccs_create(0)


@pytest.mark.parametrize("ws", [
    [small_star(n=12, depth=9, region_full=(0, 1, 2, 3), boundary=4, window=(2, 6))],
    [config2()],
    config4(64)[:12],
    [hwea(300, rounds=5, n_t=1, n_z=8, shots=5000)],
    [hwea(96, rounds=3, n_t=2, n_z=4, shots=1000, seed=7), sk_qaoa(26, n_t=1, n_z=8, shots=1000)],
], ids=["star12", "config2", "config4x12", "hwea300", "hwea96_skqaoa26"])
def test_shared_body_bit_exact(ctx, ws):
    """Brickwork plans take the one-thread-per-op body kernel; the paper's
    HWEA and SK-QAOA shapes (a few ops per moment: CX staircases and chains)
    the eight-lanes-per-op form, with 3 to 144 variants per fragment."""
    plan = ccs.ccs_build_fragments(ctx, ws)
    kw = dict(mode=ccs.CCS_SAMPLED, shots=ws[0].shots, seed_lo=SEED[0], seed_hi=SEED[1], keep_tableaus=True)
    ra = ccs.ccs_eval_variants(ctx, plan, **kw)
    rb = ccs.ccs_eval_variants(ctx, plan, per_variant_body=True, **kw)
    ma, za = ccs.ccs_recombine(ctx, plan, ra)
    mb, zb = ccs.ccs_recombine(ctx, plan, rb)
    assert np.array_equal(ma, mb) and np.array_equal(za, zb)
    rng = np.random.default_rng(1)
    checked = total = 0
    for pi in range(len(ws)):
        nf, _ = ccs.ccs_plan_counts(ctx, plan, pi)
        for f in range(nf):
            info = ccs.ccs_fragment_info_get(ctx, plan, pi, f)
            if not info["clifford"]:
                continue
            nv = info["n_variants"]
            total += nv
            for v in sorted(set([0, nv - 1] + [int(x) for x in rng.choice(nv, size=min(6, nv), replace=False)])):
                assert np.array_equal(ccs.ccs_get_tableau(ctx, ra, pi, f, v), ccs.ccs_get_tableau(ctx, rb, pi, f, v))
                assert ccs.ccs_get_outcome_space(ctx, ra, pi, f, v) == ccs.ccs_get_outcome_space(ctx, rb, pi, f, v)
                assert np.array_equal(ccs.ccs_get_counts(ctx, ra, pi, f, v), ccs.ccs_get_counts(ctx, rb, pi, f, v))
                checked += 1
    assert checked >= min(5, total)


@pytest.mark.parametrize("ws", [
    [small_star(n=12, depth=9, region_full=(0, 1, 2, 3), boundary=4, window=(2, 6), n_z=0)],
    config4(64)[:24],
], ids=["star12", "config4x24"])
def test_screen_matches_tableau_kernel(ctx, ws):
    """Variants finished by the rank screen (no tableau) carry the same
    outcome spaces and give the same marginals as the tableau kernel, which
    every variant takes when tableaus are kept."""
    plan = ccs.ccs_build_fragments(ctx, ws)
    kw = dict(mode=ccs.CCS_SAMPLED, shots=ws[0].shots, seed_lo=SEED[0], seed_hi=SEED[1])
    ra = ccs.ccs_eval_variants(ctx, plan, **kw)
    rb = ccs.ccs_eval_variants(ctx, plan, keep_tableaus=True, **kw)
    ma, _ = ccs.ccs_recombine(ctx, plan, ra)
    mb, _ = ccs.ccs_recombine(ctx, plan, rb)
    assert np.array_equal(ma, mb)
    n = 0
    for pi in range(len(ws)):
        nf, _ = ccs.ccs_plan_counts(ctx, plan, pi)
        for f in range(nf):
            info = ccs.ccs_fragment_info_get(ctx, plan, pi, f)
            if not info["clifford"]:
                continue
            for v in range(info["n_variants"]):
                assert ccs.ccs_get_outcome_space(ctx, ra, pi, f, v) == ccs.ccs_get_outcome_space(ctx, rb, pi, f, v)
                n += 1
    assert n >= 10


def test_screen_config3_all_variants(ctx):
    """Config 3's 20736 body variants: spaces from the screen equal those of
    the tableau kernel, variant by variant."""
    from workloads import config3
    w = config3()
    plan = ccs.ccs_build_fragments(ctx, [w])
    kw = dict(mode=ccs.CCS_SAMPLED, shots=w.shots, seed_lo=SEED[0], seed_hi=SEED[1])
    ra = ccs.ccs_eval_variants(ctx, plan, **kw)
    rb = ccs.ccs_eval_variants(ctx, plan, keep_tableaus=True, **kw)
    nf, _ = ccs.ccs_plan_counts(ctx, plan, 0)
    for f in range(nf):
        info = ccs.ccs_fragment_info_get(ctx, plan, 0, f)
        if info["clifford"]:
            for v in range(info["n_variants"]):
                assert ccs.ccs_get_outcome_space(ctx, ra, 0, f, v) == ccs.ccs_get_outcome_space(ctx, rb, 0, f, v), v
    ma, _ = ccs.ccs_recombine(ctx, plan, ra, precision=ccs.CCS_FP32)
    mb, _ = ccs.ccs_recombine(ctx, plan, rb, precision=ccs.CCS_FP32)
    assert np.array_equal(ma, mb)


def _with_zstrings(ws, count, seed):
    rng = np.random.default_rng(seed)
    return [Workload(w.name, w.circuit, w.cuts, w.marginal, zstrings_for(w.circuit.n_qubits, count, rng, 8),
                     w.shots, w.seed, w.regions) for w in ws]


@pytest.mark.parametrize("ws", [
    [small_star(n=12, depth=9, region_full=(0, 1, 2, 3), boundary=4, window=(2, 6))],
    [config1()],
    [config2()],
    _with_zstrings(config4(64)[:16], 24, 5),
], ids=["star12", "config1", "config2", "config4x16z"])
def test_zimages_match_tableau_kernel(ctx, ws):
    """Z-string values from the fragments' Z images (the default path: no
    tableau per variant) equal those the tableau kernel derives from each
    variant's final tableau (taken when tableaus are kept), for every
    variant, string and output subset; so do the recombined expectations."""
    plan = ccs.ccs_build_fragments(ctx, ws)
    kw = dict(mode=ccs.CCS_EXACT, seed_lo=SEED[0], seed_hi=SEED[1])
    ra = ccs.ccs_eval_variants(ctx, plan, **kw)
    rb = ccs.ccs_eval_variants(ctx, plan, keep_tableaus=True, **kw)
    ma, za = ccs.ccs_recombine(ctx, plan, ra)
    mb, zb = ccs.ccs_recombine(ctx, plan, rb)
    assert np.array_equal(za, zb) and np.array_equal(ma, mb)
    n = nonzero = 0
    for pi in range(len(ws)):
        nf, _ = ccs.ccs_plan_counts(ctx, plan, pi)
        for f in range(nf):
            info = ccs.ccs_fragment_info_get(ctx, plan, pi, f)
            if not info["clifford"] or info["n_zstrings"] == 0:
                continue
            for v in range(info["n_variants"]):
                a = ccs.ccs_get_zvals(ctx, ra, pi, f, v)
                b = ccs.ccs_get_zvals(ctx, rb, pi, f, v)
                assert np.array_equal(a, b), (pi, f, v)
                n += a.size
                nonzero += int(np.count_nonzero(a))
    assert n >= 64 and 0 < nonzero < n
