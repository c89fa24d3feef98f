"""Seeded request traces for the serving form: an open-loop Poisson stream of estimation
requests with uneven shapes, and a pool of received blocks they point at.

Each request is one frame: M in {32, 64, 128, 256} antennas, N in {255, 511, 1023, 2047}
(m-sequences of degree 8..11), L in {16, 32, 64} taps and K uniform in
1..min(floor(N / L), 16) transmitters; inter-arrival gaps are exponential at the given
rate.  Payloads: for every (M, N) a few received blocks generated with the channel model
of synth.channel (K = 1 transmitter of L = 16 taps; the estimator treats any block the
same way), stored once and shared by the requests that draw them.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import channel, mseq

M_CHOICES = (32, 64, 128, 256)
R_CHOICES = (8, 9, 10, 11)
L_CHOICES = (16, 32, 64)


@dataclass
class RequestSpec:
    rid: int
    t_arrival: float      # seconds from the start of the trace
    M: int
    N: int
    K: int
    L: int
    slot: int             # which payload of the (M, N) pool


def poisson_trace(rate_hz: float, duration_s: float, seed: int = 0, payload_slots: int = 4,
                  max_requests: int | None = None) -> list[RequestSpec]:
    rng = np.random.default_rng([seed, 7])
    n = int(rate_hz * duration_s * 1.2) + 16
    gaps = rng.exponential(1.0 / rate_hz, n)
    t = np.cumsum(gaps)
    out = []
    for i in range(n):
        if t[i] > duration_s or (max_requests is not None and len(out) >= max_requests):
            break
        M = int(rng.choice(M_CHOICES))
        r = int(rng.choice(R_CHOICES))
        N = (1 << r) - 1
        L = int(rng.choice(L_CHOICES))
        K = int(rng.integers(1, min(N // L, 16) + 1))
        out.append(RequestSpec(i, float(t[i]), M, N, K, L, int(rng.integers(0, payload_slots))))
    return out


def pilot_bits(N: int, seed: int = 0) -> np.ndarray:
    r = int(N + 1).bit_length() - 1
    if (1 << r) - 1 != N:
        raise ValueError("N must be 2^r - 1")
    return mseq.mseq_bits(r, seed)


def payload_pool(slots: int = 4, seed: int = 0, snr_db: float = 10.0):
    """{(M, N): complex64 array [slots, M, N]} of received blocks."""
    pool = {}
    for N in ((1 << r) - 1 for r in R_CHOICES):
        bits = pilot_bits(N)
        for M in M_CHOICES:
            rng = np.random.default_rng([seed, M, N])
            h = channel.channel(rng, slots, M, 1, 16)
            pool[(M, N)] = channel.received(h, bits, snr_db, rng)
    return pool
