"""C ABI on the host (no GPU): the library builds, loads and exports every
symbol of include/ccs.h; a host-only context builds plans whose fragments
agree with the oracle's independent fragmenting; bad inputs give the
documented error codes."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2303_10788_gb300 import ccs
from workloads import (Circuit, config1, config2, config3, config4, small_star, CX, H, T, random_clifford_circuit)
from oracle.cutting import fragment_circuit

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "ccs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ccs_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    ccs.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", ccs.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ccs_\w+)", out))
    declared = header_functions()
    assert declared, "no declarations parsed"
    missing = [f for f in declared if f not in exported]
    assert not missing, missing
    assert sorted(ccs.EXPORTS) == declared


def test_version():
    assert "sm_103a" in ccs.ccs_version()


@pytest.fixture(scope="module")
def hctx():
    return ccs.ccs_create(-1)


def _check_plan_against_oracle(hctx, w, problem_objs=None):
    plan = ccs.ccs_build_fragments(hctx, [w])
    frags, cuts = fragment_circuit(w.circuit, w.cuts, w.marginal)
    nf, nc = ccs.ccs_plan_counts(hctx, plan, 0)
    assert (nf, nc) == (len(frags), len(cuts))
    assert ccs.ccs_plan_cuts(hctx, plan, 0) == cuts
    for fi, f in enumerate(frags):
        info = ccs.ccs_fragment_info_get(hctx, plan, 0, fi)
        assert info["n_wires"] == f.n
        assert bool(info["clifford"]) == f.clifford
        assert info["n_variants"] == f.n_variants
        assert (info["n_qin"], info["n_qout"]) == (len(f.qin), len(f.qout))
        assert info["n_marg"] == len(f.marg)
        assert info["n_meas"] == len(f.A)
        assert info["n_slots"] == len(f.slots)
        assert ccs.ccs_fragment_wires(hctx, plan, 0, fi) == f.wires
        if f.clifford:
            # fused ops cannot outnumber gates; moments bound by gate count
            assert info["n_ops"] <= len(f.gates) and info["n_moments"] <= max(1, info["n_ops"])
    return plan


@pytest.mark.parametrize("w", [small_star(), config1(), config2(),
                               small_star(n=12, depth=9, region_full=(0, 1, 2, 3), boundary=4,
                                          window=(2, 6), n_t=3, seed=3)])
def test_fragments_match_oracle(hctx, w):
    _check_plan_against_oracle(hctx, w)


def test_fragments_match_oracle_large(hctx):
    w = config3()
    plan = _check_plan_against_oracle(hctx, w)
    body = [ccs.ccs_fragment_info_get(hctx, plan, 0, f) for f in range(5)]
    assert sorted(b["n_wires"] for b in body) == [2, 2, 2, 2, 500]
    assert max(b["n_variants"] for b in body) == 20736


def test_many_circuit_plan(hctx):
    ws = config4(16)
    plan = ccs.ccs_build_fragments(hctx, ws)
    for i, w in enumerate(ws):
        frags, cuts = fragment_circuit(w.circuit, w.cuts, w.marginal)
        assert ccs.ccs_plan_counts(hctx, plan, i) == (len(frags), len(cuts))


def _expect(hctx, probs, code):
    with pytest.raises(ccs.CCSError) as e:
        ccs.ccs_build_fragments(hctx, probs)
    assert code in str(e.value)


class _P:
    def __init__(self, circuit, cuts, marginal, zstrings=()):
        self.circuit, self.cuts, self.marginal, self.zstrings = circuit, cuts, marginal, list(zstrings)


def test_error_codes(hctx):
    c = Circuit(3)
    c.add(H, 0); c.add(CX, 0, 1); c.add(CX, 1, 2); c.add(T, 2)
    _expect(hctx, [_P(c, [(5, 1)], [0])], "INVALID_ARG")            # cut qubit out of range
    _expect(hctx, [_P(c, [(0, 99)], [0])], "INVALID_ARG")           # cut position out of range
    _expect(hctx, [_P(c, [], [7])], "INVALID_ARG")                  # marginal qubit out of range
    _expect(hctx, [_P(c, [], [0, 0])], "INVALID_ARG")               # repeated marginal qubit
    bad = Circuit(2); bad.gates.append((42, 0, -1))
    _expect(hctx, [_P(bad, [], [0])], "UNSUPPORTED_GATE")
    bad = Circuit(2); bad.gates.append((11, 0, -1))                 # first opcode past CCS_ZPOW
    _expect(hctx, [_P(bad, [], [0])], "UNSUPPORTED_GATE")
    for a in (float("nan"), float("inf"), 1e308):                   # Z^a needs a finite 2a
        bad = Circuit(2); bad.add_zpow(0, a)
        _expect(hctx, [_P(bad, [], [0])], "INVALID_ARG")
    _expect(hctx, [_P(Circuit(0), [], [])], "INVALID_ARG")          # no qubits
    huge = Circuit((1 << 24) + 1); huge.add(H, 0)                   # beyond the qubit bound
    _expect(hctx, [_P(huge, [], [0])], "INVALID_ARG")
    with pytest.raises(ccs.CCSError) as e:                          # the cut search checks it too
        ccs.ccs_cut_candidates(hctx, _P(huge, None, [0]))
    assert "INVALID_ARG" in str(e.value)
    loop = Circuit(2)                                               # both ends of the cut in one fragment
    loop.add(CX, 0, 1); loop.add(H, 0); loop.add(CX, 0, 1)
    _expect(hctx, [_P(loop, [(0, 1)], [0])], "UNSUPPORTED")
    wide = Circuit(14)
    for q in range(13):
        wide.add(CX, q, q + 1)
    wide.add(T, 0)
    _expect(hctx, [_P(wide, [], [0])], "NC_TOO_WIDE")
    many = Circuit(2)
    for _ in range(14):
        many.add(CX, 0, 1)
    _expect(hctx, [_P(many, [(0, i) for i in range(1, 14)], [0])], "TOO_MANY_CUTS")
    chain = Circuit(1025)                                           # Clifford fragment wider than 1024 wires
    for q in range(1024):
        chain.add(CX, q, q + 1)
    _expect(hctx, [_P(chain, [], [0])], "UNSUPPORTED")
    _expect(hctx, [_P(chain, [], list(range(25)))], "INVALID_ARG")  # marginal wider than 24 qubits
    idle = Circuit(14)                                              # 14 fragments: more than a problem may have
    for q in range(14):
        idle.add(H, q)
    _expect(hctx, [_P(idle, [], [0])], "UNSUPPORTED")
    idle13 = Circuit(13)                                            # 13 fragments: accepted
    for q in range(13):
        idle13.add(H, q)
    ccs.ccs_build_fragments(hctx, [_P(idle13, [], [0])])


def test_host_only_context_cannot_evaluate(hctx):
    plan = ccs.ccs_build_fragments(hctx, [small_star()])
    with pytest.raises(ccs.CCSError) as e:
        ccs.ccs_eval_variants(hctx, plan)
    assert "UNSUPPORTED" in str(e.value)


def test_batched_plan_equals_single_plans():
    """Problems planned together (on host threads) give the same fragments
    as each problem planned alone."""
    from workloads import config4
    hctx = ccs.ccs_create(-1)
    ws = config4(64)[:16]
    plan = ccs.ccs_build_fragments(hctx, ws)
    for pi, w in enumerate(ws):
        one = ccs.ccs_build_fragments(hctx, [w])
        assert ccs.ccs_plan_counts(hctx, plan, pi) == ccs.ccs_plan_counts(hctx, one, 0)
        nf, _ = ccs.ccs_plan_counts(hctx, one, 0)
        for f in range(nf):
            assert ccs.ccs_fragment_info_get(hctx, plan, pi, f) == ccs.ccs_fragment_info_get(hctx, one, 0, f)
            assert ccs.ccs_fragment_wires(hctx, plan, pi, f) == ccs.ccs_fragment_wires(hctx, one, 0, f)


def test_clifford_zpow_plans_like_its_gate(hctx):
    """Z^a with 2a an integer is planned as S^{2a}: Z^{1/2}, Z^1, Z^{-1/2}
    give the same fragments and compiled op stream sizes as S, Z, S^dagger,
    and Z^2 (the identity) stays a Clifford no-op."""
    from workloads import ZPOW, S, SDG, Z
    base = random_clifford_circuit(6, 60, seed=21)
    for a, op in ((0.5, S), (1.0, Z), (-0.5, SDG), (2.0, None)):
        cz, cg = Circuit(6, list(base.gates)), Circuit(6, list(base.gates))
        cz.gates.insert(30, (ZPOW, 2, -1, a))
        cg.gates.insert(30, (op, 2, -1) if op is not None else (S, 2, -1))
        if op is None:
            cg.gates.insert(31, (SDG, 2, -1))                       # S S^dagger: also the identity
        iz = ccs.ccs_fragment_info_get(hctx, ccs.ccs_build_fragments(hctx, [_P(cz, [], [0, 2])]), 0, 0)
        ig = ccs.ccs_fragment_info_get(hctx, ccs.ccs_build_fragments(hctx, [_P(cg, [], [0, 2])]), 0, 0)
        assert iz["clifford"] and ig["clifford"]
        if op is not None:
            assert (iz["n_ops"], iz["n_moments"]) == (ig["n_ops"], ig["n_moments"])
