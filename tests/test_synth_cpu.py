"""The synthetic input recipe, pinned directly: the exponential power-delay profile and its
unit link power, the L_nz tap model of Sec. II, the receive model y = sum over the
transmitters' shifted pilots convolved cyclically with their CIRs (brute force), the
noise variance at the stated SNR per frame, and the two shift rules."""
import math

import numpy as np

from synth import channel as C
from synth import mseq


def test_exp_pdp_unit_power_and_decay():
    w = C.exp_pdp(64, 0.3)
    assert abs(w.sum() - 1.0) < 1e-12
    assert np.allclose(w[1:] / w[:-1], math.exp(-0.3), rtol=0, atol=1e-12)


def test_channel_tap_powers_follow_the_profile():
    rng = np.random.default_rng(0)
    h = C.channel(rng, 2000, 4, 2, 16)                    # 16000 links
    p = np.mean(np.abs(h) ** 2, axis=(0, 1, 2))
    want = C.exp_pdp(16)
    n = h.shape[0] * h.shape[1] * h.shape[2]
    # |h|^2 of one tap is exponential: relative standard error 1/sqrt(n)
    assert np.all(np.abs(p / want - 1) < 5 / math.sqrt(n))
    assert abs(np.mean(np.sum(np.abs(h) ** 2, -1)) - 1.0) < 5 / math.sqrt(n)
    # circular complex Gaussian: E[h^2] = 0
    assert np.all(np.abs(np.mean(h ** 2, axis=(0, 1, 2))) < 5 * want / math.sqrt(n))


def test_lnz_model_distinct_taps_of_equal_variance():
    rng = np.random.default_rng(1)
    L, lnz = 32, 5
    h = C.channel(rng, 1000, 4, 2, L, lnz=lnz)
    nz = np.abs(h) > 0
    assert np.all(nz.sum(-1) == lnz)                       # exactly lnz distinct positions
    v = np.mean(np.abs(h[nz]) ** 2)
    assert abs(v * lnz - 1.0) < 5 / math.sqrt(nz.sum())    # each tap of variance 1/lnz
    share = nz.mean(axis=(0, 1, 2))                        # positions uniform over [0, L)
    assert np.all(np.abs(share - lnz / L) < 5 * math.sqrt(lnz / L / (nz.shape[0] * 8)))


def test_noise_free_receive_is_the_cyclic_sum():
    rng = np.random.default_rng(2)
    bits = mseq.mseq_bits(5, seed=0)
    N = bits.size
    p = mseq.bpsk(bits)
    K, L = 3, 6
    h = C.channel(rng, 2, 3, K, L)
    y = C.received(h, bits, 10.0, rng, noise=False)
    want = np.zeros((2, 3, N), dtype=np.complex128)
    for k in range(K):
        for l in range(L):
            for n in range(N):
                want[:, :, n] += h[:, :, k, l] * p[(n - l - k * L) % N]
    assert np.max(np.abs(y - want)) < 1e-5                 # complex64 output


def test_noise_variance_per_frame_snr():
    rng = np.random.default_rng(3)
    bits = mseq.mseq_bits(9, seed=0)
    h = C.channel(rng, 3, 32, 1, 4)
    snr = np.array([0.0, 10.0, 20.0])
    y = C.received(h, bits, snr, np.random.default_rng(4))
    y0 = C.received(h, bits, snr, np.random.default_rng(4), noise=False)
    w = (y - y0).astype(np.complex128)
    n = w.shape[1] * w.shape[2]
    for f in range(3):
        var = np.mean(np.abs(w[f]) ** 2)
        assert abs(var / 10 ** (-snr[f] / 10) - 1) < 5 / math.sqrt(n)
        # real and imaginary parts carry half the power each
        assert abs(np.mean(w[f].real ** 2) / np.mean(w[f].imag ** 2) - 1) < 10 / math.sqrt(n)


def test_shift_rules():
    assert list(C.shifts_kl(4, 16, 127)) == [0, 16, 32, 48]
    assert list(C.shifts_spread(4, 16, 127)) == [0, 31, 62, 93]      # k * floor(N/K), Eq. 8
