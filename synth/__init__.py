"""Seeded synthetic inputs shared by the CPU oracle, the tests and the bench.

This package holds no GEMM arithmetic: only a counter-based generator
(splitmix64, Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) and fixed maps from its 64-bit outputs to the value
distributions of the synthetic workloads.
"""
from .generators import (  # noqa: F401
    GOLDEN_GAMMA,
    BASE_SEED,
    splitmix64,
    raw_stream,
    uniform_pm1,
    integers_pm8,
    hard_magnitudes,
    log_uniform_ints,
    matrix,
    grouped_problems,
    poisson_gaps_ms,
)
