"""ORACLE — test infrastructure, not the product.

A plain, slow, obviously-correct CPU restatement of the Clifford-based
circuit-cutting method (Smith, Perlin et al., "Clifford-based Circuit Cutting
for Quantum Simulation", Sec. III-B and Sec. V): byte-per-bit CHP tableaus,
full GF(2) elimination, Philox4x32-10 written from Salmon et al. (SC'11), a
dense complex128 statevector, an FP64 recombination summed naively over the
4^k cut terms, and the maximum-likelihood correction of fragment models
(``mlcorrect``: Choi blocks, dense Hermitian eigendecomposition, simplex
projection).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import anything from here.  It shares no code with the
CUDA library (``paper_2303_10788_gb300``); both only read the seeded inputs
of ``workloads``.
"""
