"""ORACLE (test infrastructure): maximum-likelihood correction of fragment models.

Sec. V-C: before the contraction, the fragment data are turned into fragment
models that are self-consistent, which mitigates the sampling error of the
Clifford fragments' shots.  The paper states only this purpose; the method
is in its reference on maximum-likelihood fragment tomography.  The reading
implemented here:

* The model of fragment f is its Choi form, one operator per outcome o of
  its marginal wires, on the fragment's cut slots (d of them, slot order):
      J_o = 2^-d sum_P T_f(o, P) (x)_j s_j(P_j),
  s_j(P) = P^T where slot j is a quantum input, P where it is a quantum
  output.  T_f(o, P) = Tr[(x)_j s_j(P_j) J_o] gives T_f back, so J and T_f
  carry the same numbers.  For the fragment's instrument E_o (input qubits
  to output qubits, outcome o), T_f(o, P) = Tr[P_out E_o(P_in)] and J_o is
  E_o's Choi operator sum_ab |a><b| (x) E_o(|a><b|).
* Self-consistent (physical): every J_o positive semidefinite and
  sum_o Tr J_o = 2^{q_in} (trace preservation summed over the inputs; the
  finer per-input condition is not imposed).  Shot data always satisfy the
  trace condition; only positivity can fail.
* Maximum likelihood under Gaussian shot noise of equal variance in every
  T_f entry: the physical model nearest in Frobenius norm (the two norms
  agree up to the factor 2^-d).  With all blocks' eigenvalues projected
  together onto {lambda >= 0, sum = 2^{q_in}} (the Euclidean projection onto
  a scaled simplex) and each block rebuilt from its own eigenvectors -- the
  eigenvalue-projection method of Smolin, Gambetta and Smith (Phys. Rev.
  Lett. 108, 070502, 2012) applied to the block-diagonal operator.

Only tests/, the smoke check and bench.py's CPU baseline may use this module.
"""
from __future__ import annotations

import numpy as np

_PAULI = [np.eye(2, dtype=complex),
          np.array([[0, 1], [1, 0]], complex),
          np.array([[0, -1j], [1j, 0]], complex),
          np.array([[1, 0], [0, -1]], complex)]


def slot_is_input(frag):
    """Per cut slot (ascending cut id): True where the fragment has a quantum
    input on that cut."""
    ins = {c for c, _ in frag.qin}
    return [c in ins for c in frag.slots]


def slot_operators(frag, transpose_inputs=True):
    """The 4^d operators (x)_j s_j(P_j), P = sum_j P_j 4^j (T_f's Pauli index),
    slot 0 the leftmost Kronecker factor.  ``transpose_inputs=False`` drops the
    transpose at the inputs (only for tests that show the transpose matters)."""
    kinds = slot_is_input(frag)
    d = len(kinds)
    ops = []
    for P in range(4 ** d):
        op = np.ones((1, 1), complex)
        for j in range(d):
            s = _PAULI[(P >> (2 * j)) & 3]
            if kinds[j] and transpose_inputs:
                s = s.T
            op = np.kron(op, s)
        ops.append(op)
    return np.array(ops)


def choi_blocks(frag, T, transpose_inputs=True):
    """J[o] = 2^-d sum_P T[o, P] ops[P]  (complex, 2^m x 2^d x 2^d)."""
    T = np.asarray(T, np.float64)
    ops = slot_operators(frag, transpose_inputs)
    d = len(frag.slots)
    D = 1 << d
    J = T @ ops.reshape(4 ** d, D * D) / float(D)
    return J.reshape(T.shape[0], D, D)


def tensor_from_choi(frag, J):
    """T[o, P] = Re Tr[ops[P] J[o]] (the imaginary part vanishes for Hermitian J)."""
    ops = slot_operators(frag)
    d = len(frag.slots)
    D = 1 << d
    # Tr[A B] = sum_ab A[a, b] B[b, a]
    opsT = np.transpose(ops, (0, 2, 1)).reshape(4 ** d, D * D)
    return (np.asarray(J).reshape(J.shape[0], D * D) @ opsT.T).real


def project_simplex(lam, total):
    """Euclidean projection of ``lam`` onto {x >= 0, sum x = total}: the
    textbook sort-and-threshold construction.  Sort descending as u; rho is
    the largest j with u_j > (sum_{i<=j} u_i - total) / j; then
    theta = (sum_{i<=rho} u_i - total) / rho and x = max(lam - theta, 0).
    Returns (x, theta)."""
    lam = np.asarray(lam, np.float64)
    u = np.sort(lam)[::-1]
    css = np.cumsum(u)
    j = np.arange(1, len(u) + 1)
    cond = u - (css - total) / j > 0
    rho = int(np.nonzero(cond)[0][-1]) + 1
    theta = (css[rho - 1] - total) / rho
    return np.maximum(lam - theta, 0.0), theta


def ml_correct(frag, T):
    """Corrected tensor T'_f (same layout as T_f, float64) and the diagnostics
    (threshold theta, smallest eigenvalue before the correction)."""
    J = choi_blocks(frag, T)
    w, V = np.linalg.eigh(J)                      # per block, ascending
    lam, theta = project_simplex(w.ravel(), float(2 ** len(frag.qin)))
    lam = lam.reshape(w.shape)
    Jc = np.einsum("oak,ok,obk->oab", V, lam, V.conj())
    return tensor_from_choi(frag, Jc), {"theta": theta, "min_eig": float(w.min())}


def is_physical(frag, T, tol=1e-9):
    """Every Choi block positive semidefinite (smallest eigenvalue >= -tol) and
    the traces summing to 2^{q_in} within tol."""
    J = choi_blocks(frag, T)
    w = np.linalg.eigvalsh(J)
    tr = float(np.trace(J, axis1=1, axis2=2).real.sum())
    return bool(w.min() >= -tol and abs(tr - 2 ** len(frag.qin)) <= tol * max(1.0, tr))
