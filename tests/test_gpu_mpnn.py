"""The learned cut scorer on the GPU against its FP64 oracle (needs a GPU).

Forward and gradient go through the library's own kernels and are compared
with the oracle evaluated at the same FP16-rounded weights: the GPU keeps
activations and sums in FP32, so the stated tolerances are FP32 rounding
(forward 1e-4 relative, gradient 2e-3 of the largest entry).  Training by
the library's Adam kernel must fit a fixed batch, and a plan whose cut set
the trained scorer chose must give the same exact marginal as the uncut
circuit (cut-set invariance).
"""
import numpy as np
import pytest

from paper_2303_10788_gb300 import ccs
from oracle import mpnn as om
from oracle.pipeline import brute_force
from workloads import Workload, small_star

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return ccs.ccs_create(0)


def star_graphs(ctx):
    ws = [small_star(n=12, depth=9, region_full=(0, 1, 2, 3), boundary=4, window=(2, 6), seed=s) for s in (1, 2)]
    ws += [small_star(n=10, depth=8, region_full=(0, 1, 2), boundary=3, window=(2, 5), seed=3)]
    graphs = []
    for w in ws:
        for cuts, _ in ccs.ccs_cut_candidates(ctx, Workload(w.name, w.circuit, None, w.marginal, [], w.shots, w.seed))[:4]:
            graphs.append(ccs.ccs_featurize(ctx, w, cuts))
    return graphs


def oracle_inputs(batch):
    a = batch._arrays
    A = om.dense_A(a["rowptr"], a["col"], a["val"], int(batch.n_nodes))
    return a["x"].astype(np.float64), A, a["graph_off"], a["glob"].astype(np.float64)


def test_forward_and_gradient_match_oracle(ctx):
    graphs = star_graphs(ctx)
    assert len(graphs) >= 6
    b = ccs.make_batch(graphs)
    net = ccs.ccs_mpnn_create(ctx, seed=11)
    theta = ccs.ccs_mpnn_params(ctx, net).astype(np.float16).astype(np.float64)
    x, A, goff, glob = oracle_inputs(b)
    y_gpu = ccs.ccs_mpnn_forward(ctx, net, b)
    y_orc, _ = om.forward(theta, x, A, goff, glob)
    assert np.allclose(y_gpu, y_orc, rtol=1e-4, atol=1e-4 * np.abs(y_orc).max())
    t = np.linspace(-1.0, 1.0, len(graphs))
    loss_gpu, g_gpu = ccs.ccs_mpnn_gradient(ctx, net, b, t)
    loss_orc, g_orc = om.loss_and_grad(theta, x, A, goff, glob, t)
    assert loss_gpu == pytest.approx(loss_orc, rel=1e-4)
    err = np.abs(g_gpu - g_orc).max() / np.abs(g_orc).max()
    print(f"scorer gradient: max rel err {err:.2e} over {om.N_PARAMS} parameters")
    assert err < 2e-3


def test_training_fits_a_batch(ctx):
    graphs = star_graphs(ctx)
    b = ccs.make_batch(graphs)
    net = ccs.ccs_mpnn_create(ctx, seed=5)
    rng = np.random.default_rng(0)
    t = rng.normal(size=len(graphs)).astype(np.float32)
    first = ccs.ccs_mpnn_gradient(ctx, net, b, t)[0]
    for _ in range(400):
        last = ccs.ccs_mpnn_train_step(ctx, net, b, t, lr=3e-3)
    final = ccs.ccs_mpnn_gradient(ctx, net, b, t)[0]
    print(f"scorer training: loss {first:.3e} -> {final:.3e}")
    assert final < 0.1 * first


def test_learned_cut_choice_keeps_exact_results(ctx):
    w = small_star(n=12, depth=9, region_full=(0, 1, 2, 3), boundary=4, window=(2, 6), seed=2)
    search = Workload(w.name, w.circuit, None, w.marginal, [], w.shots, w.seed)
    exact, _ = brute_force(w.circuit, w.marginal)
    net = ccs.ccs_mpnn_create(ctx, seed=3)
    ccs.ccs_set_cut_model(ctx, net)
    try:
        for learned in (0, 1):
            plan = ccs.ccs_build_fragments(ctx, [search], use_learned=learned)
            res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_EXACT)
            marg, _ = ccs.ccs_recombine(ctx, plan, res)
            assert np.abs(marg - exact).max() < 1e-5, learned
    finally:
        ccs.ccs_set_cut_model(ctx, None)
