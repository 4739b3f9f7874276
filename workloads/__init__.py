"""Seeded synthetic inputs for the Clifford circuit-cutting hot path.

This package only decides *which* gates, cuts, marginal qubits, Z-strings and
random numbers make up a workload.  It holds none of the method's arithmetic
(no tableau, statevector, sampling or recombination code), so the oracle and
the CUDA path can both consume it without sharing any computation.
"""

from .circuits import (  # noqa: F401
    H, S, SDG, X, Y, Z, CX, CZ, T, TDG, ZPOW, GATE_NAMES, NQ, gate_param,
    Circuit, Region, Workload, SEED_BASE,
    random_c1_word, random_c2_word, brickwork_star,
    config1, config2, config3, config4, config5_circuit, small_star,
    random_clifford_circuit, tree_circuit, random_distributions, zstrings_for,
    t_to_s, hwea, sk_qaoa,
)
