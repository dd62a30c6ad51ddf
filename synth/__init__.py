"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

Holds configuration numbers, segment generators and the synthetic field
response table; none of the simulated method's arithmetic.
"""
from . import params, events, response  # noqa: F401
