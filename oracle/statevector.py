"""ORACLE (test infrastructure): dense complex128 statevector.

An exact statevector simulator of the kind the paper uses for non-Clifford
fragments (Sec. V-B) and as the accuracy reference (Sec. VI-C).  Amplitude
index bit q is qubit q; qubits start in |0> and outputs are measured in the
computational basis (Sec. V-B).  Gate matrices follow Sec. II: Y = -iZX,
H = (Z + X)/sqrt(2), T = Z^{1/4} = diag(1, e^{i pi/4}), and generally
Z^a = diag(1, e^{i pi a}) (Sec. II-C, Sec. VIII).
"""
from __future__ import annotations

import numpy as np

from workloads import H, S, SDG, X, Y, Z, CX, CZ, T, TDG, ZPOW, gate_param

_R2 = 1.0 / np.sqrt(2.0)
MATS = {
    H: np.array([[_R2, _R2], [_R2, -_R2]], np.complex128),
    S: np.array([[1, 0], [0, 1j]], np.complex128),
    SDG: np.array([[1, 0], [0, -1j]], np.complex128),
    X: np.array([[0, 1], [1, 0]], np.complex128),
    Y: np.array([[0, -1j], [1j, 0]], np.complex128),
    Z: np.array([[1, 0], [0, -1]], np.complex128),
    T: np.array([[1, 0], [0, np.exp(1j * np.pi / 4)]], np.complex128),
    TDG: np.array([[1, 0], [0, np.exp(-1j * np.pi / 4)]], np.complex128),
}


def zpow_matrix(a):
    """Z^a = diag(1, e^{i pi a}): Z = Z^1, S = Z^{1/2}, T = Z^{1/4}.  The
    phase has period 2 in a; a is reduced mod 2 (exactly, by fmod) first so
    that large exponents keep full precision."""
    return np.array([[1, 0], [0, np.exp(1j * np.pi * np.fmod(a, 2.0))]], np.complex128)


def apply(psi, n, op, a, b=-1, param=0.0):
    idx = np.arange(1 << n)
    if op == CX:
        ctrl = (idx >> a) & 1
        return psi[idx ^ (ctrl << b)]
    if op == CZ:
        sign = 1 - 2 * (((idx >> a) & 1) & ((idx >> b) & 1))
        return psi * sign
    U = zpow_matrix(param) if op == ZPOW else MATS[op]
    i0 = idx[((idx >> a) & 1) == 0]
    i1 = i0 | (1 << a)
    out = psi.copy()
    out[i0] = U[0, 0] * psi[i0] + U[0, 1] * psi[i1]
    out[i1] = U[1, 0] * psi[i0] + U[1, 1] * psi[i1]
    return out


def run(n, gates):
    psi = np.zeros(1 << n, np.complex128)
    psi[0] = 1.0
    for g in gates:
        psi = apply(psi, n, g[0], g[1], g[2], gate_param(g))
    return psi


def marginal(psi, n, wires):
    """Z-basis probabilities of ``wires`` (bit j of the index = wires[j])."""
    p = np.abs(psi) ** 2
    idx = np.arange(1 << n)
    y = np.zeros(1 << n, np.int64)
    for j, w in enumerate(wires):
        y |= ((idx >> w) & 1) << j
    return np.bincount(y, weights=p, minlength=1 << len(wires))


def z_expectation(psi, n, wires):
    p = np.abs(psi) ** 2
    idx = np.arange(1 << n)
    par = np.zeros(1 << n, np.int64)
    for w in wires:
        par ^= (idx >> w) & 1
    return float(np.sum(p * (1 - 2 * par)))
