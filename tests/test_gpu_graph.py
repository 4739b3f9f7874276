"""Recombination replayed from a CUDA graph equals the direct launches, bit
for bit, for every precision / tensor-core choice (needs a GPU)."""
import numpy as np
import pytest
import torch

from paper_2303_10788_gb300 import ccs
from workloads import config2, config4

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ws", [[config2()], config4(64)[:16]], ids=["config2", "config4x16"])
def test_recombine_graph_bit_identical(ws):
    ctx = ccs.ccs_create(0)
    plan = ccs.ccs_build_fragments(ctx, ws)
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=ws[0].shots, use_graph=True)
    nm = sum(1 << len(w.marginal) for w in ws)
    nz = max(1, sum(len(w.zstrings) for w in ws))
    for prec in (ccs.CCS_FP32, ccs.CCS_BF16):
        ref, zref = ccs.ccs_recombine(ctx, plan, res, precision=prec)
        for _ in range(2):
            m = torch.zeros(nm, dtype=torch.float64, device="cuda")
            z = torch.zeros(nz, dtype=torch.float64, device="cuda")
            ccs.ccs_recombine(ctx, plan, res, precision=prec, marginal_out=m, zexp_out=z, use_graph=True)
            torch.cuda.synchronize()
            assert np.array_equal(m.cpu().numpy(), ref)
            if len(zref):
                assert np.array_equal(z.cpu().numpy()[:len(zref)], zref)


@pytest.mark.parametrize("make", ["config1", "skqaoa26"])
def test_autotuned_evaluation_path_matches_default(make):
    """The autotuner may switch a small plan to the per-variant path (every
    variant simulates its whole circuit); the outcome spaces, the recombined
    marginal and the Z-string values must equal the default shared-body path
    bit for bit, directly and replayed from the evaluation graph."""
    import workloads as W
    ctx = ccs.ccs_create(0)
    if make == "config1":
        ws = [W.config1()]
    else:
        ws = [W.sk_qaoa(26, rounds=1, n_t=1, n_z=8, shots=5000, seed=W.SEED_BASE + 7)]
    plan = ccs.ccs_build_fragments(ctx, ws)
    ev = dict(mode=ccs.CCS_SAMPLED, shots=ws[0].shots, seed_lo=5, seed_hi=6)
    ref = ccs.ccs_eval_variants(ctx, plan, **ev)
    assert ccs.ccs_get_tuning(ctx, ref)[4] == 0
    m_ref, z_ref = ccs.ccs_recombine(ctx, plan, ref)
    tuned = ccs.ccs_eval_variants(ctx, plan, autotune=True, use_graph=True, **ev)
    path = ccs.ccs_get_tuning(ctx, tuned)[4]
    print(f"{make}: autotuned path = {'per-variant' if path else 'shared body'}")
    for _ in range(2):
        ccs.ccs_eval_variants(ctx, plan, res=tuned, use_graph=True, **ev)
        m, z = ccs.ccs_recombine(ctx, plan, tuned)
        assert np.array_equal(m, m_ref) and np.array_equal(z, z_ref)
    nf, _ = ccs.ccs_plan_counts(ctx, plan, 0)
    for f in range(nf):
        info = ccs.ccs_fragment_info_get(ctx, plan, 0, f)
        if info["clifford"]:
            for v in range(0, info["n_variants"], max(1, info["n_variants"] // 7)):
                assert ccs.ccs_get_outcome_space(ctx, tuned, 0, f, v) == ccs.ccs_get_outcome_space(ctx, ref, 0, f, v)
