"""Seeded synthetic channels and received pilot blocks.

System model (Sec. II, Eq. 2 and Eq. 6/9 with the cyclic-shift multiplexing of
Sec. II-B): K transmitters share one length-N m-sequence pilot p, transmitter k
using the cyclic shift k*L.  After cyclic-prefix removal antenna m of frame f sees

    y_{f,m}[n] = sum_k sum_{l<L} h[f,m,k,l] * p[(n - l - k*L) mod N] + w[n]

i.e. the circulant pilot matrix applied to the zero-padded stacked CIR
x[j] = h[k, l] at j = k*L + l (a circular convolution of x with p).

Channel: every (f, m, k) link has L complex Gaussian taps with an exponential
power-delay profile, power proportional to exp(-decay * l), normalised to unit total
power.  Noise: circular complex Gaussian of variance 10^(-SNR/10) (each
transmitter's received power is one).  The paper's own sparse-tap model (L_nz taps
placed uniformly inside L) is available through `lnz`.

The received block is computed in float64 and returned as complex64, the dtype the
estimator consumes.  This module is an input generator only: the circular
convolution here is the channel (transmit side), not the estimator.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.fft as sfft

from . import mseq


def exp_pdp(L: int, decay: float = 0.3) -> np.ndarray:
    w = np.exp(-decay * np.arange(L, dtype=np.float64))
    return w / w.sum()


def channel(rng: np.random.Generator, F: int, M: int, K: int, L: int,
            decay: float = 0.3, lnz: int | None = None) -> np.ndarray:
    """Complex128 CIRs h[F, M, K, L].

    lnz=None: exponential power-delay profile over all L taps (unit power per link).
    lnz=int: the paper's model -- lnz distinct tap positions drawn uniformly in [0, L)
    per link, each tap of variance 1/lnz (unit expected power per link).
    """
    g = rng.standard_normal((F, M, K, L, 2))
    h = (g[..., 0] + 1j * g[..., 1]) / np.sqrt(2.0)
    if lnz is None:
        h *= np.sqrt(exp_pdp(L, decay))
    else:
        if not 1 <= lnz <= L:
            raise ValueError("need 1 <= lnz <= L")
        keys = rng.random((F, M, K, L))
        rank = np.argsort(np.argsort(keys, axis=-1), axis=-1)
        h = np.where(rank < lnz, h / np.sqrt(lnz), 0.0)
    return h


def stacked_cir(h: np.ndarray, N: int) -> np.ndarray:
    """x[..., j] = h[..., k, l] at j = k*L + l, zero for j >= K*L (length N)."""
    *lead, K, L = h.shape
    if K * L > N:
        raise ValueError("K*L must not exceed N")
    x = np.zeros((*lead, N), dtype=np.complex128)
    x[..., : K * L] = h.reshape(*lead, K * L)
    return x


def received(h: np.ndarray, bits: np.ndarray, snr_db, rng: np.random.Generator,
             chunk_rows: int = 8192, noise: bool = True) -> np.ndarray:
    """Received complex64 blocks Y[F, M, N] for CIRs h[F, M, K, L] and pilot bits.

    snr_db: scalar or per-frame array of length F.  noise=False gives the noise-free
    block (the SNR is then ignored).
    """
    F, M, K, L = h.shape
    N = bits.size
    p = mseq.bpsk(bits)
    Pf = sfft.fft(p)
    x = h.reshape(F * M, K * L)
    y = np.empty((F * M, N), dtype=np.complex64)
    snr = np.broadcast_to(np.asarray(snr_db, dtype=np.float64), (F,))
    sigma = np.sqrt(10.0 ** (-snr / 10.0) / 2.0)
    for r0 in range(0, F * M, chunk_rows):
        r1 = min(F * M, r0 + chunk_rows)
        xs = np.zeros((r1 - r0, N), dtype=np.complex128)
        xs[:, : K * L] = x[r0:r1]
        ys = sfft.ifft(sfft.fft(xs, axis=1, workers=-1) * Pf, axis=1, workers=-1)
        if noise:
            g = rng.standard_normal((r1 - r0, N, 2))
            s = sigma[np.arange(r0, r1) // M][:, None]
            ys = ys + s * (g[..., 0] + 1j * g[..., 1])
        y[r0:r1] = ys
    return y.reshape(F, M, N)


def shifts_kl(K: int, L: int, N: int) -> np.ndarray:
    """Cyclic shift of transmitter k: k*L (contiguous lags)."""
    return np.arange(K) * L


def shifts_spread(K: int, L: int, N: int) -> np.ndarray:
    """Cyclic shift of transmitter k spread evenly over the sequence: k*floor(N/K)."""
    return np.arange(K) * (N // K)


def received_with_cp(h: np.ndarray, bits: np.ndarray, snr_db, rng: np.random.Generator,
                     cp_len: int, shifts=None, noise: bool = True) -> np.ndarray:
    """Received blocks of cp_len + N samples, cyclic prefix included (Sec. II-A, Fig. 1).

    Transmitter k sends its cyclically shifted pilot s_k[n] = p[(n - shift_k) mod N] preceded
    by its last cp_len samples; the channel acts by LINEAR convolution with h[f,m,k,:]; the
    receiver keeps the first cp_len + N samples.  With L <= cp_len + 1 the samples after
    the prefix equal the circular model of `received`.
    """
    F, M, K, L = h.shape
    N = bits.size
    p = mseq.bpsk(bits)
    sh = shifts_kl(K, L, N) if shifts is None else np.asarray(shifts)
    T = cp_len + N
    y = np.zeros((F, M, T), dtype=np.complex128)
    for k in range(K):
        s = p[(np.arange(N) - sh[k]) % N]
        tx = np.concatenate([s[N - cp_len:], s]) if cp_len else s
        for l in range(L):
            y[..., l:] += h[..., k, l][..., None] * tx[None, None, : T - l]
    if noise:
        snr = np.broadcast_to(np.asarray(snr_db, dtype=np.float64), (F,))
        sigma = np.sqrt(10.0 ** (-snr / 10.0) / 2.0)[:, None, None]
        g = rng.standard_normal((F, M, T, 2))
        y = y + sigma * (g[..., 0] + 1j * g[..., 1])
    return y.astype(np.complex64)


@dataclass(frozen=True)
class Workload:
    """One synthetic estimation workload (shapes of the paper's sweeps)."""
    name: str
    r: int          # LFSR degree, N = 2^r - 1
    M: int          # receive antennas
    K: int          # multiplexed transmitters (cyclic shifts k*L)
    L: int          # CIR taps
    F: int          # frames per launch
    snr_db: tuple   # SNRs; frame f uses snr_db[f % len(snr_db)]
    seed: int = 0

    @property
    def N(self) -> int:
        return (1 << self.r) - 1

    def frame_snr(self) -> np.ndarray:
        s = np.asarray(self.snr_db, dtype=np.float64)
        return s[np.arange(self.F) % s.size]


# The five synthetic workloads: tiny plain FP32, paper-like scale, precision form,
# differentiation form (shapes; the serving form is in synth.serving).
SMALL = Workload("n127_m8_k2_l16_f1", r=7, M=8, K=2, L=16, F=1, snr_db=(10.0,), seed=0)
PAPER_SCALE = Workload("n1023_m64_k8_l64_f128", r=10, M=64, K=8, L=64, F=128,
                       snr_db=(0.0, 10.0, 20.0), seed=1)
PRECISION = Workload("n4095_m128_k16_l128_f512", r=12, M=128, K=16, L=128, F=512,
                     snr_db=(0.0, 10.0, 20.0, 30.0), seed=2)
DIFFERENTIATION = Workload("n1023_m64_k8_l64_f64", r=10, M=64, K=8, L=64, F=64,
                           snr_db=(10.0,), seed=3)
WORKLOADS = {w.name: w for w in (SMALL, PAPER_SCALE, PRECISION, DIFFERENTIATION)}


def make_received(w: Workload, frames: int | None = None, first: int = 0):
    """(bits, Y) for frames [first, first + frames) of workload w, without keeping h."""
    F = w.F if frames is None else frames
    bits = mseq.mseq_bits(w.r, w.seed)
    snr = w.frame_snr()
    Y = np.empty((F, w.M, w.N), dtype=np.complex64)
    for i in range(F):
        f = first + i
        rng = np.random.default_rng([w.seed, f])
        h = channel(rng, 1, w.M, w.K, w.L)
        Y[i] = received(h, bits, snr[f % snr.size], rng)[0]
    return bits, Y


def make(w: Workload, frames: int | None = None, noise: bool = True):
    """(bits, h, Y) for workload w, optionally only its first `frames` frames.

    The channel of frame f depends only on (seed, f), so a prefix of frames is the
    same data as the corresponding frames of the full workload.
    """
    F = w.F if frames is None else frames
    bits = mseq.mseq_bits(w.r, w.seed)
    hs, ys = [], []
    snr = w.frame_snr()
    for f in range(F):
        rng = np.random.default_rng([w.seed, f])
        h = channel(rng, 1, w.M, w.K, w.L)
        hs.append(h)
        ys.append(received(h, bits, snr[f], rng, noise=noise))
    return bits, np.concatenate(hs), np.concatenate(ys)
