"""Contexts on the library's own stream-ordered memory pool (created without
an allocator): plans built on two host threads, each with its own context,
then evaluated and recombined step after step on a third give exactly the
marginal and Z values of a context on torch's allocator (same kernels, same
Philox shots); freed results return to the pool; destroying a context trims
the pool without disturbing the live plans of another."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_2303_10788_gb300 import ccs
from workloads import config2

pytestmark = pytest.mark.gpu
EV = dict(mode=ccs.CCS_SAMPLED, shots=1000, seed_lo=0x99, seed_hi=0x42)


def test_pool_contexts_match_torch_allocator():
    w = config2()
    ref = ccs.ccs_create(0)
    plan = ccs.ccs_build_fragments(ref, [w])
    res = ccs.ccs_eval_variants(ref, plan, **EV)
    want, wz = ccs.ccs_recombine(ref, plan, res)

    main = ccs.ccs_create(0, torch_allocator=False)
    builders = [ccs.ccs_create(0, torch_allocator=False) for _ in range(2)]
    with ThreadPoolExecutor(2) as ex:
        plans = list(ex.map(lambda c: ccs.ccs_build_fragments(c, [w]), builders))
    for p in plans:
        for _ in range(3):
            r = ccs.ccs_eval_variants(main, p, **EV)
            m, z = ccs.ccs_recombine(main, p, r)
            assert np.array_equal(m, want) and np.array_equal(z, wz)
            del r
    # the first builder's plan goes, then its context (the pool is trimmed);
    # the other builder's plan still evaluates to the same values
    first, other = plans
    del plans, p, first
    builders[0].close()
    r = ccs.ccs_eval_variants(main, other, use_graph=True, **EV)
    m, z = ccs.ccs_recombine(main, other, r, use_graph=True)
    assert np.array_equal(m, want) and np.array_equal(z, wz)
