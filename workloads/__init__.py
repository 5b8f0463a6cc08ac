"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and
the benchmark.

This package draws random exponent sets and coefficients only.  It holds none
of the multiplication arithmetic: no Kronecker coding, no products, no
canonicalisation of results.  Every draw comes from a counter-based SplitMix64
stream (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; constants as published by Vigna), so the same seed
gives the same inputs on x86 and Arm hosts.
"""
from .synth import (  # noqa: F401
    Rng, Poly, PSeries, total_degree_tuples,
    dense_total_degree, dense_box, mp_sparse, poisson_random, random_poly, random_pseries,
    workload_cfg1, workload_cfg2, workload_cfg3, workload_cfg4, batch_mix, fateman,
    arrival_times,
)
