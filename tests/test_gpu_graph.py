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
