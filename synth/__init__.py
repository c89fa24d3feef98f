"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

Input generation only (pilot bits, channels, received blocks, request traces): no
estimator arithmetic lives here.
"""
from . import channel, mseq  # noqa: F401
