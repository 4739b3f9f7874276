"""Clifford-specific stitching (Sec. IX) against strong simulation.

CCS_STITCH forms each Clifford hub's contraction operand in closed form from
its variants' outcome spaces (no shots, no per-variant distribution) and the
contraction skips the operand rows that vanish identically.  Its results
must equal the oracle's exact mode (each Clifford variant 2^-rank on its
outcome space, Sec. V-C) within the 1e-5 absolute bound, and its operand
rows must equal the GPU's own exact-mode operand (formed from dense
distributions) bit for bit where nonzero and be exactly zero where flagged.
Config 3 and the config-4 circuits compare with stored oracle results
(tests/golden/exact_marginals.npz, written by make_golden.py from the
oracle's outcome spaces).
"""
import os

import numpy as np
import pytest

from paper_2303_10788_gb300 import ccs
from workloads import Workload, config1, config2, config3, config4, small_star, t_to_s
from oracle.pipeline import evaluate_workload, uncut_clifford

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "exact_marginals.npz")
TOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    return ccs.ccs_create(0)


def _stitched(ctx, ws, **kw):
    plan = ccs.ccs_build_fragments(ctx, ws)
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_STITCH, **kw)
    return plan, res


@pytest.mark.parametrize("make", [lambda: small_star(seed=3), lambda: small_star(n=10, depth=8, seed=8), config1,
                                  config2])
def test_stitch_matches_oracle_exact(ctx, make):
    w = make()
    plan, res = _stitched(ctx, [w], use_graph=True)
    m, z = ccs.ccs_recombine(ctx, plan, res, use_graph=True)
    orc = evaluate_workload(w, mode="exact", keep_tableaus=False)
    assert np.abs(m - orc.marginal).max() < TOL
    if len(w.zstrings):
        assert np.abs(z - orc.zexp).max() < TOL
    # the operand rows: nonzero ones equal the exact-mode operand bit for
    # bit, flagged ones are zero there too
    res_e = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_EXACT)
    nf, _ = ccs.ccs_plan_counts(ctx, plan, 0)
    hub = max(range(nf), key=lambda f: ccs.ccs_fragment_info_get(ctx, plan, 0, f)["n_slots"])
    qs, qe = ccs.ccs_get_operand(ctx, res, 0, hub), ccs.ccs_get_operand(ctx, res_e, 0, hub)
    assert np.array_equal(qs, qe)
    zero_rows = int((np.abs(qe).max(axis=0) == 0).sum())
    print(f"{w.name}: {zero_rows} of {qe.shape[1]} hub operand rows vanish; "
          f"max|err| {np.abs(m - orc.marginal).max():.2e}")


def test_stitch_keep_tableaus_and_bf16(ctx):
    w = config2()
    plan, res = _stitched(ctx, [w])
    m, z = ccs.ccs_recombine(ctx, plan, res)
    res_k = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_STITCH, keep_tableaus=True)
    mk, zk = ccs.ccs_recombine(ctx, plan, res_k)
    assert np.abs(m - mk).max() < 1e-12 and np.abs(z - zk).max() < 1e-12
    m16, _ = ccs.ccs_recombine(ctx, plan, res, precision=ccs.CCS_BF16)
    assert np.abs(m16 - m).max() < 1e-3


def test_stitch_config3_full_size(ctx):
    g = np.load(GOLD)
    plan, res = _stitched(ctx, [config3()], use_graph=True)
    m32, _ = ccs.ccs_recombine(ctx, plan, res, use_graph=True)
    m16, _ = ccs.ccs_recombine(ctx, plan, res, precision=ccs.CCS_BF16, use_graph=True)
    e32, e16 = np.abs(m32 - g["config3"]).max(), np.abs(m16 - g["config3"]).max()
    print(f"config3 stitched vs FP64 oracle (exact): fp32 {e32:.2e}, bf16 {e16:.2e}")
    assert e32 < TOL and e16 < 2e-4


def test_stitch_config3_t_to_s(ctx):
    """All T -> S: the circuit is Clifford, so the stitched marginal must be
    one uncut tableau's closed form (2^-rank on its outcome space)."""
    w = config3()
    c = t_to_s(w.circuit)
    ws = Workload("c3s", c, w.cuts, w.marginal, [], w.shots, w.seed)
    plan, res = _stitched(ctx, [ws])
    m, _ = ccs.ccs_recombine(ctx, plan, res)
    cf, _ = uncut_clifford(c, w.marginal)
    assert np.abs(m - cf).max() < TOL


def test_stitch_config4_batch(ctx):
    g = np.load(GOLD)
    ws = config4(256)
    plan, res = _stitched(ctx, ws, use_graph=True)
    m, _ = ccs.ccs_recombine(ctx, plan, res, use_graph=True)
    offs = np.concatenate([[0], np.cumsum([1 << len(w.marginal) for w in ws])])
    worst = 0.0
    for i, ci in enumerate(g["config4_circuits"]):
        ci = int(ci)
        worst = max(worst, np.abs(m[offs[ci]:offs[ci + 1]] - g["config4"][i]).max())
    print(f"config4 stitched vs FP64 oracle (exact), circuits {list(g['config4_circuits'])}: {worst:.2e}")
    assert worst < TOL
