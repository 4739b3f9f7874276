"""Contraction of any fragment topology (Sec. V-C: one tensor per fragment,
one index per cut), not only stars.

Blocks of three wires joined in a tree: each child block's first wire takes
one gate from its parent block and is cut right after it, so the fragments
follow the tree.  Chains and branched trees of four and five fragments have
no fragment touching every cut; the library contracts them with the general
kernel (each output summed over the whole cut index from all fragment
tensors).  Exact mode must equal the oracle and the uncut statevector,
sampled mode the oracle on the same Philox shots, within 1e-5 (marginals and
Z-string values); BF16 within 1e-2; two halves of the cut index sum to the
whole.
"""
import numpy as np
import pytest

from paper_2303_10788_gb300 import ccs
from workloads import Workload, tree_circuit
from oracle.pipeline import brute_force, evaluate

pytestmark = pytest.mark.gpu
SEED = (0x2468, 0x1357)
# (name, parent of each child block, T count, Z-strings spanning blocks)
SHAPES = [
    ("chain4", [0, 1, 2], 2, [[0, 1, 11], [1, 10]]),
    ("branch4", [0, 0, 1], 1, [[7, 11], [1, 6, 8], [0, 6, 8]]),
    ("chain5", [0, 1, 2, 3], 2, [[3, 10, 12], [10, 12], [2, 14]]),
    ("branch5", [0, 0, 1, 1], 3, [[1, 4, 5], [1, 6, 8], [0, 13]]),
]


@pytest.fixture(scope="module")
def ctx():
    return ccs.ccs_create(0)


@pytest.mark.parametrize("name,parents,n_t,zs", SHAPES)
def test_tree_topology_matches_oracle(ctx, name, parents, n_t, zs):
    c, cuts = tree_circuit(parents, 16, n_t, seed=1)
    n = c.n_qubits
    marg = [0, 2, 4, n - 3, n - 1]
    w = Workload(name, c, cuts, marg, zs, 512, 3)
    plan = ccs.ccs_build_fragments(ctx, [w])
    nf, nc = ccs.ccs_plan_counts(ctx, plan, 0)
    assert nf == len(parents) + 1 and nc == len(parents)
    slots = [ccs.ccs_fragment_info_get(ctx, plan, 0, f)["n_slots"] for f in range(nf)]
    assert max(slots) < nc, "expected a fragment graph that is not a star"

    bf, bz = brute_force(c, marg, zs)
    assert np.abs(bz).max() > 0.5       # Z-strings with a non-zero value
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_EXACT)
    m, z = ccs.ccs_recombine(ctx, plan, res)
    assert np.abs(m - bf).max() < 1e-5 and np.abs(z - bz).max() < 1e-5
    m16, _ = ccs.ccs_recombine(ctx, plan, res, precision=ccs.CCS_BF16)
    assert np.abs(m16 - bf).max() < 1e-2
    K = 4 ** nc
    a, _ = ccs.ccs_recombine(ctx, plan, res, k_range=(0, K // 2))
    b, _ = ccs.ccs_recombine(ctx, plan, res, k_range=(K // 2, K))
    assert np.abs(a + b - m).max() < 1e-7

    res_s = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=w.shots,
                                  seed_lo=SEED[0], seed_hi=SEED[1])
    ms, zsv = ccs.ccs_recombine(ctx, plan, res_s)
    orc = evaluate(c, cuts, marg, zs, mode="sampled", shots=w.shots, seed_lo=SEED[0], seed_hi=SEED[1])
    assert np.abs(ms - orc.marginal).max() < 1e-5 and np.abs(zsv - orc.zexp).max() < 1e-5
