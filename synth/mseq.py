"""Seeded m-sequence (maximal-length PN sequence) pilots.

The paper transmits a length-N PN sequence as the pilot (Sec. II-A, Eq. 1) but does
not say how it is generated.  Here it is the output of a Fibonacci linear-feedback
shift register of degree r (N = 2^r - 1) whose characteristic polynomial is chosen,
by seed, among the primitive polynomials of that degree:

* polynomials f(x) = x^r + sum_{i<r} c_i x^i with c_0 = 1 are enumerated in
  increasing integer encoding (bit i of the integer = c_i, bit r set);
* f is primitive iff the class of x has multiplicative order exactly 2^r - 1 in
  GF(2)[x]/(f); those are kept, and index ``seed % count`` is taken;
* the register starts in state (a_0..a_{r-1}) = (1, 0, ..., 0) and obeys
  a_{t+r} = sum_i c_i a_{t+i} (mod 2); the sequence bits are b[n] = a_n.

Any other nonzero start state gives a cyclic shift of the same sequence; since the
same bits are used at the transmitter and receiver that choice does not change an
estimate.  BPSK mapping (bit 0 -> +1, bit 1 -> -1) is applied by the consumers.

This module is an input generator only: it holds none of the estimator's arithmetic.
"""
from __future__ import annotations

import functools

import numpy as np


def _prime_factors(n: int) -> list[int]:
    out, d = [], 2
    while d * d <= n:
        if n % d == 0:
            out.append(d)
            while n % d == 0:
                n //= d
        d += 1
    if n > 1:
        out.append(n)
    return out


def _gf2_mulmod(a: int, b: int, f: int, r: int) -> int:
    """Product of two GF(2) polynomials (ints, bit i = coeff of x^i) modulo f (degree r)."""
    acc = 0
    while b:
        if b & 1:
            acc ^= a
        b >>= 1
        a <<= 1
        if a >> r & 1:
            a ^= f
    return acc


def _gf2_powmod_x(e: int, f: int, r: int) -> int:
    """x^e mod f."""
    result, base = 1, 2
    while e:
        if e & 1:
            result = _gf2_mulmod(result, base, f, r)
        base = _gf2_mulmod(base, base, f, r)
        e >>= 1
    return result


def is_primitive(f: int, r: int) -> bool:
    """True iff polynomial f (degree r, constant term 1) is primitive over GF(2)."""
    if f >> r != 1 or not (f & 1):
        return False
    order = (1 << r) - 1
    if _gf2_powmod_x(order, f, r) != 1:
        return False
    return all(_gf2_powmod_x(order // q, f, r) != 1 for q in _prime_factors(order))


@functools.lru_cache(maxsize=None)
def primitive_polynomials(r: int) -> tuple[int, ...]:
    """All primitive polynomials of degree r, increasing integer encoding."""
    if r < 2 or r > 24:
        raise ValueError("degree r must be in [2, 24]")
    cands = ((1 << r) | mid | 1 for mid in range(0, 1 << r, 2))
    return tuple(f for f in cands if is_primitive(f, r))


def lfsr_bits(f: int, r: int, length: int) -> np.ndarray:
    """First `length` output bits of the Fibonacci LFSR with characteristic polynomial f."""
    taps = [i for i in range(r) if f >> i & 1]
    a = np.zeros(length + r, dtype=np.uint8)
    a[0] = 1
    for t in range(length):
        v = 0
        for i in taps:
            v ^= int(a[t + i])
        a[t + r] = v
    return a[:length].copy()


def mseq_bits(r: int, seed: int = 0) -> np.ndarray:
    """The seeded m-sequence of degree r as a uint8 array of N = 2^r - 1 bits."""
    polys = primitive_polynomials(r)
    f = polys[seed % len(polys)]
    return lfsr_bits(f, r, (1 << r) - 1)


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """Pack bits LSB-first into uint32 words: bit n lives in word n // 32, bit n % 32."""
    bits = np.asarray(bits, dtype=np.uint8).ravel()
    nw = (bits.size + 31) // 32
    padded = np.zeros(nw * 32, dtype=np.uint64)
    padded[: bits.size] = bits
    weights = (np.uint64(1) << np.arange(32, dtype=np.uint64))
    return (padded.reshape(nw, 32) * weights).sum(axis=1).astype(np.uint32)


def unpack_bits(words: np.ndarray, n: int) -> np.ndarray:
    words = np.asarray(words, dtype=np.uint32)
    idx = np.arange(n)
    return ((words[idx // 32] >> (idx % 32).astype(np.uint32)) & 1).astype(np.uint8)


def bpsk(bits: np.ndarray) -> np.ndarray:
    """Bit 0 -> +1.0, bit 1 -> -1.0 (float64)."""
    return 1.0 - 2.0 * np.asarray(bits, dtype=np.float64)
