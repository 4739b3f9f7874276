"""ccs_recombine_noalloc: recombination for callers that cannot allocate device
memory when they need the result (its scratch is a fixed array inside the
library).  Checked through the C ABI against ccs_recombine on two calls in a
row, and for its size limit.  Collected last on purpose."""
import numpy as np
import pytest

from paper_2303_10788_gb300 import ccs
from workloads import Region, Workload, brickwork_star, config1, config2

pytestmark = pytest.mark.gpu

TOL = 1e-5     # the recombined-probability tolerance of the parity tests


@pytest.fixture(scope="module")
def ctx():
    return ccs.ccs_create(0)


@pytest.mark.parametrize("make", [config1, config2])
def test_noalloc_matches_recombine_twice(ctx, make):
    import torch
    w = make()
    plan = ccs.ccs_build_fragments(ctx, [w])
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=w.shots, seed_lo=3, seed_hi=4)
    ref_m, ref_z = ccs.ccs_recombine(ctx, plan, res)
    for _ in range(2):
        m = torch.full((1 << len(w.marginal),), -1.0, dtype=torch.float64, device="cuda")
        z = torch.full((len(w.zstrings),), -7.0, dtype=torch.float64, device="cuda")
        ccs.ccs_recombine_noalloc(ctx, plan, res, m, z)
        torch.cuda.synchronize()
        assert np.abs(m.cpu().numpy() - ref_m).max() < TOL
        assert np.abs(z.cpu().numpy() - ref_z).max() < TOL


def test_noalloc_rejects_plans_beyond_its_scratch(ctx):
    import torch
    # four leaves carrying the whole 12-qubit marginal and 8 cuts: the
    # Kronecker operand alone is 4^8 x 2^12 floats (1 GiB) > 8 MiB
    regs = [Region([0, 1, 2], 3, 2, 6, [0, 1, 2], 1),
            Region([10, 11, 12], 13, 2, 6, [10, 11, 12], 1),
            Region([20, 21, 22], 23, 2, 6, [20, 21, 22], 1),
            Region([30, 31, 32], 33, 2, 6, [30, 31, 32], 1)]
    c, cuts = brickwork_star(40, 9, regs, seed=1)
    w = Workload("big", c, cuts, [0, 1, 2, 10, 11, 12, 20, 21, 22, 30, 31, 32], [], 256, 1)
    plan = ccs.ccs_build_fragments(ctx, [w])
    nf, nc = ccs.ccs_plan_counts(ctx, plan, 0)
    slots = [ccs.ccs_fragment_info_get(ctx, plan, 0, f)["n_slots"] for f in range(nf)]
    assert nc == 8 and max(slots) == 8          # a star: the body carries every cut
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=256)
    m = torch.zeros(1 << 12, dtype=torch.float64, device="cuda")
    with pytest.raises(ccs.CCSError) as e:
        ccs.ccs_recombine_noalloc(ctx, plan, res, m)
    assert "UNSUPPORTED" in str(e.value) and "scratch" in str(e.value)
