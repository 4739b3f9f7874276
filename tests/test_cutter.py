"""Cut search on the host (no GPU).

Any valid cut set reproduces the uncut circuit exactly (the cut identity), so
the oracle's exact-mode result on the searched cuts is pinned to brute force;
on star-shaped workloads the search never needs more cuts than the planted
partition.
"""
import numpy as np
import pytest

from paper_2303_10788_gb300 import ccs
from workloads import config1, config2, config3, config4, small_star, random_clifford_circuit
from oracle.pipeline import evaluate, brute_force


class _P:
    def __init__(self, circuit, marginal, zstrings=()):
        self.circuit, self.cuts, self.marginal, self.zstrings = circuit, None, marginal, list(zstrings)


@pytest.fixture(scope="module")
def hctx():
    return ccs.ccs_create(-1)


@pytest.mark.parametrize("w", [small_star(n=10, depth=8, region_full=(0, 1, 2), boundary=3, window=(2, 5),
                                          n_t=3, seed=2),
                               small_star(n=12, depth=7, region_full=(0,), boundary=1, window=(2, 4),
                                          n_t=2, seed=8)])
def test_searched_cuts_are_exact(hctx, w):
    cands = ccs.ccs_cut_candidates(hctx, _P(w.circuit, w.marginal, w.zstrings), max_nc_width=4)
    assert cands and all(c1[1] <= c2[1] for c1, c2 in zip(cands, cands[1:]))
    bf, bz = brute_force(w.circuit, w.marginal, w.zstrings)
    for cuts, _ in cands[:3]:
        r = evaluate(w.circuit, cuts, w.marginal, w.zstrings, mode="exact")
        assert max(f.n for f in r.fragments if not f.clifford) <= 4
        assert np.abs(r.marginal - bf).max() < 1e-12
        assert np.abs(r.zexp - bz).max() < 1e-12


def test_random_circuits_with_t(hctx):
    for seed in range(4):
        c = random_clifford_circuit(7, 50, seed + 40, t_count=2)
        marg = [0, 3, 6]
        cands = ccs.ccs_cut_candidates(hctx, _P(c, marg), max_nc_width=5)
        bf, _ = brute_force(c, marg)
        r = evaluate(c, cands[0][0], marg, mode="exact")
        assert np.abs(r.marginal - bf).max() < 1e-12


def test_search_matches_planted_partition(hctx):
    ws = [config1(), config2(), config3()] + config4(12)
    for w in ws:
        plan = ccs.ccs_build_fragments(hctx, [_P(w.circuit, w.marginal)])
        nf, nc = ccs.ccs_plan_counts(hctx, plan, 0)
        assert nc <= len(w.cuts), w.name
        infos = [ccs.ccs_fragment_info_get(hctx, plan, 0, f) for f in range(nf)]
        assert all(i["n_wires"] <= 10 for i in infos if not i["clifford"])


def test_clifford_circuit_needs_no_cuts(hctx):
    c = random_clifford_circuit(30, 200, 3)
    assert ccs.ccs_cut_candidates(hctx, _P(c, [0, 1]))[0][0] == []
