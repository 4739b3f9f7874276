"""Maximum-likelihood correction of fragment models on the GPU (Sec. V-C)
against the FP64 oracle (``oracle.mlcorrect``) on the same Philox shots.

Per fragment the corrected tensor T'_f must match the oracle's element by
element, and the recombined marginal of the corrected models the oracle's
contraction of its corrected tensors.  Bars (complex64 Jacobi against FP64
``eigh``): T'_f within 4 N 2^-24 of the oracle relative to max(1, max |T_f|),
N = 2^(d+1) the real dimension of a 2^d x 2^d complex Choi block (the
rounding of an FP32 eigendecomposition and of the rebuild grows like N eps
times the block's norm: 2e-6 at d = 2, 3e-5 at d = 6); marginals within
1e-5.  Cases cover fragments with 1 to 6 cut slots: stars (the hub operand
stored by preparation at its inputs, as int16 count sums; one hub with 5
slots, one with 6) and a branched tree (general contraction, T_f read
directly).
"""
import numpy as np
import pytest

from paper_2303_10788_gb300 import ccs
from workloads import Workload, Region, brickwork_star, small_star, config1, config2, tree_circuit, t_to_s
from oracle.cutting import recombine
from oracle.mlcorrect import ml_correct, is_physical
from oracle.pipeline import evaluate

pytestmark = pytest.mark.gpu
SEED = (0x5EED, 0x0A11)


def t_bar(d):
    return 4.0 * (2 << d) * 2.0 ** -24


def three_region_star():
    """A hub with six cut slots (three regions, each cut in and out)."""
    regs = [Region([0], 1, 2, 6, [0, 1], 1), Region([7], 8, 3, 7, [7, 8], 1), Region([15], 14, 2, 5, [15, 14], 1)]
    c, cuts = brickwork_star(16, 10, regs, 77)
    return Workload("star3x", c, cuts, [0, 7, 15, 3, 5, 10, 12], [], 256, 77, regs)


def five_slot_star():
    """A hub with five cut slots: the third region runs to the circuit's end
    (an input cut only)."""
    regs = [Region([0], 1, 2, 6, [0, 1], 1), Region([7], 8, 3, 7, [7, 8], 1), Region([15], 14, 2, 10, [15, 14], 1)]
    c, cuts = brickwork_star(16, 10, regs, 78)
    return Workload("star5s", c, cuts, [0, 7, 15, 3, 5, 10, 12], [], 256, 78, regs)


def tree4():
    c, cuts = tree_circuit([0, 1, 1], 12, 2, seed=4)
    return Workload("tree4", c, cuts, [0, 2, 4, 6, c.n_qubits - 1], [], 128, 4)


CASES = {
    "star8": lambda: small_star(),
    "config1": config1,
    "config2": config2,
    "star3x": three_region_star,
    "star5s": five_slot_star,
    "tree4": tree4,
}
SHOTS = {"star8": 64, "config1": 96, "config2": 128, "star3x": 256, "star5s": 256, "tree4": 128}


@pytest.fixture(scope="module")
def ctx():
    return ccs.ccs_create(0)


def _oracle(w, shots, mode="sampled"):
    return evaluate(w.circuit, w.cuts, w.marginal, (), mode=mode, shots=shots, seed_lo=SEED[0], seed_hi=SEED[1])


@pytest.mark.parametrize("name", list(CASES))
def test_ml_correction_matches_oracle(ctx, name):
    w = CASES[name]()
    shots = SHOTS[name]
    orc = _oracle(w, shots)
    k = orc.meta["k"]
    want = [ml_correct(f, T)[0] if f.clifford else T for f, T in zip(orc.fragments, orc.tensors)]
    want_m = recombine(orc.fragments, want, k, len(w.marginal))

    plan = ccs.ccs_build_fragments(ctx, [w])
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=shots, seed_lo=SEED[0], seed_hi=SEED[1],
                                use_graph=True)
    raw, _ = ccs.ccs_recombine(ctx, plan, res)
    assert np.abs(raw - orc.marginal).max() < 1e-5          # the data the correction starts from
    ccs.ccs_ml_correct(ctx, plan, res, ccs.CCS_ML_SAMPLED)
    worst = 0.0
    for fi, (f, Tw) in enumerate(zip(orc.fragments, want)):
        got = ccs.ccs_get_tensor(ctx, res, 0, fi).astype(np.float64)
        err = np.abs(got - Tw).max() / max(1.0, np.abs(Tw).max())
        worst = max(worst, err)
        assert err < t_bar(len(f.slots)), (fi, len(f.slots), err)
        if f.clifford:
            assert is_physical(f, got, tol=1e-4)
    m, _ = ccs.ccs_recombine(ctx, plan, res, use_graph=True)
    print(f"{name}: worst T' error {worst:.2e}, marginal {np.abs(m - want_m).max():.2e}")
    assert np.abs(m - want_m).max() < 1e-5
    assert m.min() > -1e-5                                  # no negative quasi-probability left
    mb, _ = ccs.ccs_recombine(ctx, plan, res, precision=ccs.CCS_BF16)
    assert np.abs(mb - want_m).max() < 1e-2
    # a second correction reads the corrected (FP32) operands: the corrected
    # models are physical, so it leaves them where they are
    ccs.ccs_ml_correct(ctx, plan, res, ccs.CCS_ML_SAMPLED)
    m2, _ = ccs.ccs_recombine(ctx, plan, res, use_graph=True)
    assert np.abs(m2 - want_m).max() < 1e-5
    # the next evaluation brings back the raw data (and the int16 hub operand)
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=shots, seed_lo=SEED[0], seed_hi=SEED[1],
                                use_graph=True, res=res)
    again, _ = ccs.ccs_recombine(ctx, plan, res, use_graph=True)
    assert np.abs(again - raw).max() < 1e-7


@pytest.mark.parametrize("name", ["config2", "star3x", "tree4"])
def test_exact_models_are_fixed_points(ctx, name):
    """CCS_ML_ALL on an exact result: every model is physical already, so the
    tensors and the marginal come back unchanged within FP32 rounding."""
    w = CASES[name]()
    orc = _oracle(w, 0, mode="exact")
    plan = ccs.ccs_build_fragments(ctx, [w])
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_EXACT)
    before, _ = ccs.ccs_recombine(ctx, plan, res)
    # the default selection has nothing to correct in an exact result: every
    # tensor (the hub's folded on request) stays the evaluation's
    ccs.ccs_ml_correct(ctx, plan, res, ccs.CCS_ML_SAMPLED)
    for fi, (f, T) in enumerate(zip(orc.fragments, orc.tensors)):
        assert np.abs(ccs.ccs_get_tensor(ctx, res, 0, fi) - T).max() / max(1.0, np.abs(T).max()) < 1e-5
    ccs.ccs_ml_correct(ctx, plan, res, ccs.CCS_ML_ALL)
    for fi, (f, T) in enumerate(zip(orc.fragments, orc.tensors)):
        got = ccs.ccs_get_tensor(ctx, res, 0, fi)
        assert np.abs(got - T).max() / max(1.0, np.abs(T).max()) < t_bar(len(f.slots))
    after, _ = ccs.ccs_recombine(ctx, plan, res)
    assert np.abs(after - orc.marginal).max() < 1e-5 and np.abs(after - before).max() < 1e-5


def test_ml_batch_of_circuits(ctx):
    """Several problems in one plan (fragments of every slot count in one
    launch group set): each problem's corrected marginal equals the oracle's."""
    ws = [small_star(seed=s, shots=64) for s in (2, 3)] + [three_region_star(), tree4()]
    plan = ccs.ccs_build_fragments(ctx, ws)
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=64, seed_lo=SEED[0], seed_hi=SEED[1])
    ccs.ccs_ml_correct(ctx, plan, res)
    m, _ = ccs.ccs_recombine(ctx, plan, res)
    off = 0
    for ci, w in enumerate(ws):
        orc = evaluate(w.circuit, w.cuts, w.marginal, (), mode="sampled", shots=64, seed_lo=SEED[0],
                       seed_hi=SEED[1], circuit_id=ci)
        want = [ml_correct(f, T)[0] if f.clifford else T for f, T in zip(orc.fragments, orc.tensors)]
        want_m = recombine(orc.fragments, want, orc.meta["k"], len(w.marginal))
        n = 1 << len(w.marginal)
        assert np.abs(m[off:off + n] - want_m).max() < 1e-5, w.name
        off += n


def test_ml_rejections(ctx):
    w = three_region_star()
    plan = ccs.ccs_build_fragments(ctx, [w])
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_STITCH)
    with pytest.raises(ccs.CCSError, match="INVALID_ARG"):
        ccs.ccs_ml_correct(ctx, plan, res)
    with pytest.raises(ccs.CCSError, match="INVALID_ARG"):
        ccs.ccs_ml_correct(ctx, plan, res, 7)
    from workloads import config3
    w3 = config3()
    plan3 = ccs.ccs_build_fragments(ctx, [w3])
    res3 = ccs.ccs_eval_variants(ctx, plan3, mode=ccs.CCS_SAMPLED, shots=256)
    with pytest.raises(ccs.CCSError, match="UNSUPPORTED"):     # the hub has 8 cut slots
        ccs.ccs_ml_correct(ctx, plan3, res3)


def test_cut_free_fragment(ctx):
    """A Clifford circuit without cuts: one fragment, no cut slots, 1 x 1
    Choi blocks (its sampled marginal, already a probability vector), so the
    correction leaves it unchanged; with a cut-bearing problem beside it in
    the same plan the blocks of both slot counts are corrected in one call."""
    w0 = small_star()
    w = Workload("cliff", t_to_s(w0.circuit), [], w0.marginal, [], 256, 1)
    ws = [w, small_star(seed=3, shots=256)]
    plan = ccs.ccs_build_fragments(ctx, ws)
    res = ccs.ccs_eval_variants(ctx, plan, mode=ccs.CCS_SAMPLED, shots=256, seed_lo=SEED[0], seed_hi=SEED[1])
    raw, _ = ccs.ccs_recombine(ctx, plan, res)
    ccs.ccs_ml_correct(ctx, plan, res)
    m, _ = ccs.ccs_recombine(ctx, plan, res)
    n0 = 1 << len(w.marginal)
    assert np.abs(m[:n0] - raw[:n0]).max() < 1e-6
    orc = evaluate(ws[1].circuit, ws[1].cuts, ws[1].marginal, (), mode="sampled", shots=256, seed_lo=SEED[0],
                   seed_hi=SEED[1], circuit_id=1)
    want = [ml_correct(f, T)[0] if f.clifford else T for f, T in zip(orc.fragments, orc.tensors)]
    want_m = recombine(orc.fragments, want, orc.meta["k"], len(ws[1].marginal))
    assert np.abs(m[n0:] - want_m).max() < 1e-5
