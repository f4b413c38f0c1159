"""CPU oracle for GFD validation — TEST INFRASTRUCTURE ONLY.

Used by the tests, the smoke check and the benchmark's CPU-baseline leg; never by
the product path. See oracle/oracle.c for what it computes.
"""
from .oracle import OracleGraph, build_oracle, validate, oracle_available
from .bruteforce import brute_force

__all__ = ["OracleGraph", "build_oracle", "validate", "oracle_available", "brute_force"]
