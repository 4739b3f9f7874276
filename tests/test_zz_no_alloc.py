"""ccs_recombine_noalloc: recombination for callers that cannot allocate device
memory when they need the result (its scratch is a fixed array inside the
library).  Checked through the C ABI against ccs_recombine on two calls in a
row, in FP32 and BF16, on plans that contract leaf by leaf (no scratch) and
on a plan whose contraction runs through the fixed scratch (the leaves'
Kronecker operand and the split-K partials); on a chain of fragments; a large plan, then a small one,
then the large one again; and for its size limit.  Collected last on
purpose."""
import numpy as np
import pytest

from paper_2303_10788_gb300 import ccs
from workloads import Region, Workload, brickwork_star, config1, config2, tree_circuit

pytestmark = pytest.mark.gpu

TOL = 1e-5     # the recombined-probability tolerance of the parity tests


@pytest.fixture(scope="module")
def ctx():
    return ccs.ccs_create(0)


def scratch_star():
    """A 24-qubit star with four 2-wire leaves (8 cuts, 4^8 cut terms) and a
    7-bit hub marginal: its contraction is a GEMM over the cut index whose
    Kronecker operand (4^8 x 16 floats) and partials fit the fixed scratch."""
    regs = [Region([q], q + 1, 2, 6, [q, q + 1], 1) for q in (0, 6, 12, 18)]
    c, cuts = brickwork_star(24, 9, regs, seed=5)
    marg = [0, 6, 12, 18, 3, 4, 9, 10, 15, 16, 21]
    return Workload("scratch_star", c, cuts, marg, [[3, 9], [0, 4, 21]], 1024, 5)


def _evaluated(ctx, w):
    plan = ccs.ccs_build_fragments(ctx, [w])
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=w.shots, seed_lo=3, seed_hi=4)
    return plan, res


def _noalloc_twice(ctx, plan, res, w, precision):
    import torch
    ref_m, ref_z = ccs.ccs_recombine(ctx, plan, res, precision=precision, tensor_cores=False)
    for _ in range(2):
        m = torch.full((1 << len(w.marginal),), -1.0, dtype=torch.float64, device="cuda")
        z = torch.full((max(1, len(w.zstrings)),), -7.0, dtype=torch.float64, device="cuda")
        ccs.ccs_recombine_noalloc(ctx, plan, res, m, z, precision=precision)
        torch.cuda.synchronize()
        assert np.abs(m.cpu().numpy() - ref_m).max() < TOL
        if len(w.zstrings):
            assert np.abs(z.cpu().numpy()[:len(w.zstrings)] - ref_z).max() < TOL


@pytest.mark.parametrize("precision", [ccs.CCS_FP32, ccs.CCS_BF16])
@pytest.mark.parametrize("make", [config1, config2])
def test_noalloc_matches_recombine_twice(ctx, make, precision):
    w = make()
    plan, res = _evaluated(ctx, w)
    _noalloc_twice(ctx, plan, res, w, precision)


@pytest.mark.parametrize("precision", [ccs.CCS_FP32, ccs.CCS_BF16])
def test_noalloc_through_its_scratch_large_small_large(ctx, precision):
    w_big, w_small = scratch_star(), config1()
    nf, nc = ccs.ccs_plan_counts(ctx, ccs.ccs_build_fragments(ctx, [w_big]), 0)
    assert nc == 8
    big, small = _evaluated(ctx, w_big), _evaluated(ctx, w_small)
    _noalloc_twice(ctx, *big, w_big, precision)
    _noalloc_twice(ctx, *small, w_small, precision)
    _noalloc_twice(ctx, *big, w_big, precision)


@pytest.mark.parametrize("precision", [ccs.CCS_FP32, ccs.CCS_BF16])
def test_noalloc_non_star_plan(ctx, precision):
    # a chain of four fragments: no fragment carries every cut
    c, cuts = tree_circuit([0, 1, 2], 16, 2, seed=1)
    w = Workload("chain4", c, cuts, [0, 2, 4, 9, 11], [[0, 1, 11], [1, 10]], 512, 3)
    plan, res = _evaluated(ctx, w)
    nf, nc = ccs.ccs_plan_counts(ctx, plan, 0)
    assert max(ccs.ccs_fragment_info_get(ctx, plan, 0, f)["n_slots"] for f in range(nf)) < nc
    _noalloc_twice(ctx, plan, res, w, precision)


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
