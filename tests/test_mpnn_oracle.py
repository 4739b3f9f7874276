"""Pins of the cut scorer's FP64 oracle and of the host featurizer (CPU only).

The oracle's backward is checked against central finite differences of its
forward; the forward against a hand-computed case on an asymmetric A (a
transposed A fails it), the all-zero-weight closed form, and node
permutation invariance.
"""
import numpy as np
import pytest

from oracle import mpnn as om

rng = np.random.default_rng(7)


def random_graphs(sizes, rng):
    xs, rps, cols, vals, goff = [], [0], [], [], [0]
    for n in sizes:
        adj = np.zeros((n, n))
        for _ in range(2 * n):
            a, b = rng.integers(0, n, 2)
            if a != b:
                adj[a, b] += 1
                adj[b, a] += 1
        deg = adj.sum(1)
        base = goff[-1]
        for r in range(n):
            for c in range(n):
                if adj[r, c]:
                    cols.append(base + c)
                    vals.append(adj[r, c] / deg[r])
            rps.append(len(cols))
        xs.append(rng.normal(size=(n, om.IN)))
        goff.append(base + n)
    N = goff[-1]
    A = om.dense_A(np.array(rps), np.array(cols), np.array(vals), N)
    return np.concatenate(xs), A, np.array(goff), rng.normal(size=(len(sizes), om.GLOB))


def test_gradient_matches_central_differences():
    x, A, goff, glob = random_graphs([5, 7, 3], rng)
    theta = rng.normal(size=om.N_PARAMS) * 0.3
    t = rng.normal(size=3)
    loss, g = om.loss_and_grad(theta, x, A, goff, glob, t)
    idx = rng.choice(om.N_PARAMS, size=300, replace=False)
    # every block of the layout gets probed
    idx = np.unique(np.concatenate([idx, [o for o, _ in om.SHAPES.values()]]))
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (om.loss_and_grad(tp, x, A, goff, glob, t)[0] - om.loss_and_grad(tm, x, A, goff, glob, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def _set(theta, name, idx, value):
    o, shape = om.SHAPES[name]
    theta[o + np.ravel_multi_index(idx, shape)] = value


def test_hand_computed_path_graph():
    # path 0-1-2: A = D^-1 Adj = [[0,1,0],[.5,0,.5],[0,1,0]] (not symmetric)
    rowptr, col, val = np.array([0, 1, 3, 4]), np.array([1, 0, 2, 1]), np.array([1.0, 0.5, 0.5, 1.0])
    A = om.dense_A(rowptr, col, val, 3)
    x = np.zeros((3, om.IN))
    x[:, 0] = [1.0, 2.0, 5.0]
    theta = np.zeros(om.N_PARAMS)
    _set(theta, "W_in", (0, 0), 1.0)
    for l in range(om.LAYERS):
        _set(theta, f"Wn{l}", (0, 0), 1.0)
    _set(theta, "W_r1", (0, 0), 1.0)
    _set(theta, "w_r2", (0,), 1.0)
    _set(theta, "b_r2", (0,), 0.25)
    # h0 = [1,2,5]; A h0 = [2,3,2]; A^2 h0 = [3,2,3]; A^3 h0 = [2,3,2]; mean 7/3
    y, _ = om.forward(theta, x, A, np.array([0, 3]), np.zeros((1, om.GLOB)))
    assert y[0] == pytest.approx(7.0 / 3.0 + 0.25, abs=1e-12)


def test_zero_weights_closed_form():
    x, A, goff, glob = random_graphs([4, 6], rng)
    theta = np.zeros(om.N_PARAMS)
    b_r1 = rng.normal(size=om.HID)
    w_r2 = rng.normal(size=om.HID)
    o, _ = om.SHAPES["b_r1"]
    theta[o:o + om.HID] = b_r1
    o, _ = om.SHAPES["w_r2"]
    theta[o:o + om.HID] = w_r2
    _set(theta, "b_r2", (0,), -0.5)
    y, _ = om.forward(theta, x, A, goff, glob)
    assert np.allclose(y, np.maximum(b_r1, 0) @ w_r2 - 0.5, atol=1e-12)


def test_node_permutation_invariance():
    x, A, goff, glob = random_graphs([9], rng)
    theta = rng.normal(size=om.N_PARAMS) * 0.3
    y, _ = om.forward(theta, x, A, goff, glob)
    p = rng.permutation(9)
    y2, _ = om.forward(theta, x[p], A[np.ix_(p, p)], goff, glob)
    assert np.allclose(y, y2, atol=1e-12)


def test_featurize_host_graph():
    from paper_2303_10788_gb300 import ccs
    from workloads import small_star
    ctx = ccs.ccs_create(-1)
    w = small_star(n=12, depth=9, region_full=(0, 1, 2, 3), boundary=4, window=(2, 6))
    g = ccs.ccs_featurize(ctx, w, w.cuts)
    n = w.circuit.n_qubits
    assert g.x.shape == (n, 8) and g.rowptr[-1] == len(g.col)
    # rows of A = D^-1 Adj sum to 1 on every qubit that has a neighbour
    for q in range(n):
        a, b = g.rowptr[q], g.rowptr[q + 1]
        if b > a:
            assert g.val[a:b].sum() == pytest.approx(1.0, abs=1e-6)
    # val_t[e] is the entry of the reverse edge
    lookup = {(q, int(g.col[e])): g.val[e] for q in range(n) for e in range(g.rowptr[q], g.rowptr[q + 1])}
    for q in range(n):
        for e in range(g.rowptr[q], g.rowptr[q + 1]):
            assert g.val_t[e] == pytest.approx(lookup[(int(g.col[e]), q)])
    # per-qubit cut counts and the number of cuts in the globals
    cuts_per_q = np.bincount([c[0] for c in w.cuts], minlength=n)
    assert np.array_equal(g.x[:, 5], cuts_per_q)
    assert g.glob[0] == pytest.approx(len(w.cuts) / 8)
    assert np.all(g.x[:, 0] == 1.0)
