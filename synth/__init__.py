"""Seeded synthetic workloads shared by the tests, the oracle driver and bench.py.

This module draws random numbers only. It holds none of the verification
arithmetic: no forward pass, no digit decoding, no coverage logic. Both the
CUDA path and the CPU oracle receive the arrays it returns as plain inputs.
"""
from .gen import (  # noqa: F401
    splitmix64,
    uniform01,
    normal,
    randint,
    distinct,
    make_net,
    make_query,
    make_queries,
    make_pairs,
    WORKLOADS,
    workload,
    proposal_candidates,
)
