"""ORACLE (test infrastructure): the learned cut scorer in FP64 numpy.

Same network and parameter layout as the library's scorer:
  h0 = relu(W_in x + b_in); h_{l+1} = relu(Ws_l h_l + Wn_l (A h_l) + b_l);
  r = mean over the graph's nodes of h3; z = relu(W_r1 [r, glob] + b_r1);
  y = w_r2 . z + b_r2; loss = mean (y - t)^2.
Written straight from those definitions: dense forward and analytic
backward (chain rule through each relu, the mean and A), pinned by central
finite differences in the tests.
"""
from __future__ import annotations

import numpy as np

IN, GLOB, HID, LAYERS = 8, 8, 64, 3
R = HID + GLOB


def layout():
    shapes, off = {}, 0
    def add(name, shape):
        nonlocal off
        size = int(np.prod(shape))
        shapes[name] = (off, shape)
        off += size
    add("W_in", (HID, IN)); add("b_in", (HID,))
    for l in range(LAYERS):
        add(f"Ws{l}", (HID, HID)); add(f"Wn{l}", (HID, HID)); add(f"b{l}", (HID,))
    add("W_r1", (HID, R)); add("b_r1", (HID,)); add("w_r2", (HID,)); add("b_r2", (1,))
    return shapes, off


SHAPES, N_PARAMS = layout()


def unpack(theta):
    return {k: np.asarray(theta[o:o + int(np.prod(s))], np.float64).reshape(s) for k, (o, s) in SHAPES.items()}


def dense_A(rowptr, col, val, n):
    A = np.zeros((n, n))
    for r in range(n):
        for e in range(rowptr[r], rowptr[r + 1]):
            A[r, col[e]] += val[e]
    return A


def forward(theta, x, A, graph_off, glob):
    P = unpack(theta)
    relu = lambda v: np.maximum(v, 0.0)
    H = [relu(x @ P["W_in"].T + P["b_in"])]
    AH = []
    for l in range(LAYERS):
        AH.append(A @ H[l])
        H.append(relu(H[l] @ P[f"Ws{l}"].T + AH[l] @ P[f"Wn{l}"].T + P[f"b{l}"]))
    G = len(graph_off) - 1
    Rm = np.stack([H[-1][graph_off[g]:graph_off[g + 1]].mean(axis=0) for g in range(G)])
    RG = np.concatenate([Rm, glob], axis=1)
    Z = relu(RG @ P["W_r1"].T + P["b_r1"])
    y = Z @ P["w_r2"] + P["b_r2"][0]
    return y, dict(H=H, AH=AH, RG=RG, Z=Z, P=P)


def loss_and_grad(theta, x, A, graph_off, glob, target):
    y, c = forward(theta, x, A, graph_off, glob)
    P, H, AH, RG, Z = c["P"], c["H"], c["AH"], c["RG"], c["Z"]
    G = len(y)
    loss = float(np.mean((y - target) ** 2))
    g = {k: np.zeros(s) for k, (_, s) in SHAPES.items()}
    dy = 2.0 * (y - target) / G
    g["w_r2"] = Z.T @ dy
    g["b_r2"] = np.array([dy.sum()])
    dZ = np.outer(dy, P["w_r2"]) * (Z > 0)
    g["W_r1"] = dZ.T @ RG
    g["b_r1"] = dZ.sum(axis=0)
    dRG = dZ @ P["W_r1"]
    dH = np.zeros_like(H[-1])
    for gi in range(G):
        a, b = graph_off[gi], graph_off[gi + 1]
        dH[a:b] = dRG[gi, :HID] / (b - a)
    for l in reversed(range(LAYERS)):
        dP = dH * (H[l + 1] > 0)
        g[f"Ws{l}"] = dP.T @ H[l]
        g[f"Wn{l}"] = dP.T @ AH[l]
        g[f"b{l}"] = dP.sum(axis=0)
        dH = dP @ P[f"Ws{l}"] + A.T @ (dP @ P[f"Wn{l}"])
    dP = dH * (H[0] > 0)
    g["W_in"] = dP.T @ x
    g["b_in"] = dP.sum(axis=0)
    flat = np.zeros(N_PARAMS)
    for k, (o, s) in SHAPES.items():
        flat[o:o + int(np.prod(s))] = g[k].ravel()
    return loss, flat
