"""Pins of the FP64 oracle (and of the synthetic inputs it is fed) to facts that the
paper and the mathematics fix -- none of them re-derives the oracle's own formula.

* m-sequences: period, balance, two-valued autocorrelation (Eq. 1), the textbook table
  of primitive polynomials and the closed-form count phi(2^r - 1) / r;
* estimator: three independent forms agree on tiny inputs (brute-force loop, Toeplitz
  product, DFT correlation); the noise-free closed form h + (h - S)/N implied by
  Eq. 1-3; the full-lag circulant identity P^T P = (N+1) I - 1 1^T; the golden delta
  channel; sign / linearity invariants; the noise statistics;
* adjoint: torch float64 autograd, central finite differences and the dot-product
  (adjointness) identity;
* quantisers: torch's own CPU casts and hand-picked tie cases;
* MAE (Eq. 12) on a hand-computed case.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import pn_oracle as O
from synth import channel as C
from synth import mseq as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _phi(n):
    out, m, d = n, n, 2
    while d * d <= m:
        if m % d == 0:
            while m % d == 0:
                m //= d
            out -= out // d
        d += 1
    if m > 1:
        out -= out // m
    return out


def _read_golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            rows[k.strip()] = v.split()
    return rows


# ------------------------------------------------------------------ m-sequences


def test_primitive_polynomials_textbook_table():
    g = _read_golden("primitive_polynomials.txt")
    for r, polys in g.items():
        assert S.primitive_polynomials(int(r)) == tuple(int(x) for x in polys)


@pytest.mark.parametrize("r", range(2, 13))
def test_primitive_polynomial_count_closed_form(r):
    assert len(S.primitive_polynomials(r)) == _phi((1 << r) - 1) // r


@pytest.mark.parametrize("r", [3, 4, 5, 6, 7])
def test_primitivity_equals_brute_force_period(r):
    # brute force: a polynomial is primitive iff its LFSR from a nonzero state has
    # period exactly 2^r - 1
    N = (1 << r) - 1
    for mid in range(0, 1 << r, 2):
        f = (1 << r) | mid | 1
        b = S.lfsr_bits(f, r, 2 * N + r)
        period = next(t for t in range(1, 2 * N) if np.array_equal(b[t:t + N], b[:N]))
        assert (period == N) == S.is_primitive(f, r), (r, f, period)


@pytest.mark.parametrize("r,seed", [(3, 0), (5, 4), (7, 0), (7, 11), (10, 1), (12, 2)])
def test_mseq_period_balance_autocorrelation(r, seed):
    N = (1 << r) - 1
    b = S.mseq_bits(r, seed)
    assert b.size == N
    assert int(b.sum()) == (N + 1) // 2                       # balance
    p = 1 - 2 * b.astype(np.int64)
    R = np.array([int(np.dot(p, np.roll(p, -n))) for n in range(N)])
    assert R[0] == N and np.all(R[1:] == -1)                  # Eq. 1 (unnormalised)


def test_pack_unpack_roundtrip():
    b = S.mseq_bits(10, 3)
    w = S.pack_bits(b)
    assert w.dtype == np.uint32 and w.size == 32
    assert np.array_equal(S.unpack_bits(w, b.size), b)
    assert (int(w[0]) & 1) == b[0] and ((int(w[1]) >> 3) & 1) == b[35]


# ------------------------------------------------------------------- estimator


def _small_case(r, M, K, L, F, seed, snr=10.0, noise=True):
    w = C.Workload("t", r=r, M=M, K=K, L=L, F=F, snr_db=(snr,), seed=seed)
    return C.make(w, noise=noise)


@pytest.mark.parametrize("r,M,K,L,F", [(3, 2, 1, 3, 1), (4, 3, 3, 5, 2), (5, 2, 2, 7, 1),
                                       (7, 2, 2, 16, 1), (7, 1, 1, 127, 1)])
def test_three_oracle_forms_agree(r, M, K, L, F):
    bits, _, Y = _small_case(r, M, K, L, F, seed=r)
    H1 = O.estimate_direct(Y, bits, K, L)
    H2 = O.estimate(Y, bits, K, L)
    H3 = O.estimate_fft(Y, bits, K, L)
    scale = np.abs(H1).max()
    assert np.abs(H2 - H1).max() <= 1e-12 * scale
    assert np.abs(H3 - H1).max() <= 1e-12 * scale


def test_golden_delta_channel():
    g = _read_golden("delta_channel_n7.txt")
    bits = np.array([int(x) for x in g["bits"]], dtype=np.uint8)
    d = int(g["delay"][0])
    exp = np.array([float(Fraction(x)) for x in g["expected"]])
    p = 1.0 - 2.0 * bits
    y = np.roll(p, d)[None, None, :]                 # y[n] = p[(n - d) mod N]
    H = O.estimate(y, bits, 1, 7)[0, 0, 0]
    assert np.abs(H - exp).max() <= 1e-15


@pytest.mark.parametrize("r,M,K,L", [(7, 8, 2, 16), (10, 4, 8, 64), (6, 3, 4, 15), (5, 2, 31, 1)])
def test_noise_free_closed_form(r, M, K, L):
    # Eq. 1-3 with the shifts k*L: H_hat[j] = x[j] + (x[j] - S)/N, S = sum of all taps
    bits, h, Y = _small_case(r, M, K, L, 2, seed=7, noise=False)
    N = bits.size
    H = O.estimate(Y, bits, K, L)
    x = h.reshape(2, M, K * L)
    Ssum = x.sum(axis=-1, keepdims=True)
    want = x + (x - Ssum) / N
    # Y was rounded to complex64 by the generator: allow that rounding only
    tol = 4 * np.finfo(np.float32).eps * np.abs(Y).max()
    assert np.abs(H.reshape(2, M, K * L) - want).max() <= tol
    # exact inversion of the leakage term
    Hs = H.reshape(2, M, K * L)
    Sh = Hs.sum(axis=-1, keepdims=True) * N / (N + 1 - K * L)
    assert np.abs((N * Hs + Sh) / (N + 1) - x).max() <= 2 * tol


@pytest.mark.parametrize("r", [3, 5, 7, 9])
def test_full_lag_circulant_identity(r):
    b = S.mseq_bits(r, 1)
    N = b.size
    P = O.pilot_matrix(O.pilot_symbols(b), N)
    assert np.array_equal(P.T @ P, (N + 1) * np.eye(N) - np.ones((N, N)))


def test_circulant_first_rows_eq2():
    # Eq. 2: first row [s0, s_{N-1}, ..., s1], second row [s1, s0, s_{N-1}, ..., s2]
    s = np.arange(1, 8, dtype=np.float64)
    P = O.pilot_matrix(s, 7)
    assert list(P[0]) == [1, 7, 6, 5, 4, 3, 2]
    assert list(P[1]) == [2, 1, 7, 6, 5, 4, 3]


def test_sign_and_linearity_invariants():
    bits, _, Y = _small_case(7, 4, 2, 16, 2, seed=5)
    H = O.estimate(Y, bits, 2, 16)
    # the same sign-flipped pilot at transmitter and receiver leaves H_hat unchanged
    bits_f = 1 - bits
    Yf = -Y.astype(np.complex128)   # received block of the flipped pilot, same channel
    assert np.abs(O.estimate(Yf, bits_f, 2, 16) - H).max() <= 1e-12
    assert np.abs(O.estimate(2.5 * Y.astype(np.complex128), bits, 2, 16) - 2.5 * H).max() <= 1e-12


def test_rejects_aliasing_shapes():
    Y = np.zeros((1, 1, 7), np.complex64)
    with pytest.raises(ValueError):
        O.estimate(Y, np.zeros(7, np.uint8), 2, 4)        # K*L > N (Eq. 7)


def test_noise_statistics():
    # estimate error against the noise-free estimate is CN(0, sigma^2/N) per lag
    r, M, K, L, snr = 7, 64, 2, 16, 0.0
    bits, h, Y = _small_case(r, M, K, L, 4, seed=11, snr=snr, noise=True)
    _, _, Y0 = _small_case(r, M, K, L, 4, seed=11, noise=False)
    N = bits.size
    e = O.estimate(Y, bits, K, L) - O.estimate(Y0, bits, K, L)
    var = np.mean(np.abs(e) ** 2)
    want = 10 ** (-snr / 10) / N
    n = e.size
    assert abs(var / want - 1) < 5 / math.sqrt(n)
    # distinct lags are correlated with covariance -sigma^2/N^2
    ee = e.reshape(-1, K * L)
    cov01 = np.mean(ee[:, 0] * np.conj(ee[:, 1])).real
    assert abs(cov01 - (-want / N)) < 6 * want / math.sqrt(ee.shape[0])


def test_error_floor_shrinks_with_pn_length():
    # Sec. IV-A: at high SNR the remaining error is the -1/N leakage, smaller for longer PN
    floors = []
    for r in (7, 9, 11):
        bits, h, Y = _small_case(r, 4, 2, 16, 1, seed=2, noise=False)
        floors.append(O.mae(O.estimate(Y, bits, 2, 16), h))
    assert floors[0] > floors[1] > floors[2]


# --------------------------------------------------------------------- adjoint


def _relaxed_case(seed=0, F=2, M=3, N=31, K=2, L=5):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((F, M, N)) + 1j * rng.standard_normal((F, M, N))
    theta = rng.standard_normal(N)
    Ht = rng.standard_normal((F, M, K, L)) + 1j * rng.standard_normal((F, M, K, L))
    return Y, theta, Ht


def _loss(Y, theta, Ht, K, L):
    H = O.estimate_real_pilot(Y, np.tanh(theta), K, L)
    return float(np.mean(np.abs(H - Ht) ** 2))


def test_adjoint_matches_torch_autograd_fp64():
    torch = pytest.importorskip("torch")
    K, L = 2, 5
    Y, theta, Ht = _relaxed_case()
    F, M, N = Y.shape
    G = 2 * (O.estimate_real_pilot(Y, np.tanh(theta), K, L) - Ht) / Ht.size
    dY, dp = O.adjoint(G, Y, np.tanh(theta), K, L)

    Yt = torch.tensor(Y, dtype=torch.complex128, requires_grad=True)
    tt = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    p = torch.tanh(tt)
    idx = (torch.arange(N)[:, None] - torch.arange(K * L)[None, :]) % N
    P = p[idx].to(torch.complex128)
    H = (Yt.reshape(F * M, N) @ P / N).reshape(F, M, K, L)
    loss = (H - torch.tensor(Ht)).abs().pow(2).mean()
    loss.backward()
    assert np.abs(Yt.grad.numpy() - dY).max() <= 1e-12
    dth = dp * (1 - np.tanh(theta) ** 2)
    assert np.abs(tt.grad.numpy() - dth).max() <= 1e-12


def test_adjoint_central_differences():
    K, L, eps = 2, 5, 1e-3
    Y, theta, Ht = _relaxed_case(seed=1)
    G = 2 * (O.estimate_real_pilot(Y, np.tanh(theta), K, L) - Ht) / Ht.size
    dY, dp = O.adjoint(G, Y, np.tanh(theta), K, L)
    dth = dp * (1 - np.tanh(theta) ** 2)
    for q in range(0, theta.size, 5):
        e = np.zeros_like(theta)
        e[q] = eps
        fd = (_loss(Y, theta + e, Ht, K, L) - _loss(Y, theta - e, Ht, K, L)) / (2 * eps)
        assert abs(fd - dth[q]) <= 1e-6 * max(1.0, abs(fd))
    for (f, m, n) in [(0, 0, 0), (1, 2, 17), (0, 1, 30)]:
        for d in (1.0, 1j):
            E = np.zeros_like(Y)
            E[f, m, n] = eps * d
            fd = (_loss(Y + E, theta, Ht, K, L) - _loss(Y - E, theta, Ht, K, L)) / (2 * eps)
            g = dY[f, m, n].real if d == 1.0 else dY[f, m, n].imag
            assert abs(fd - g) <= 1e-7 * max(1.0, abs(fd))


def test_adjoint_dot_product_identity():
    # Re <G, A(Y)> = Re <A*(G), Y> for the linear map A(Y) = Y P / N
    rng = np.random.default_rng(3)
    F, M, N, K, L = 2, 2, 63, 3, 7
    Y = rng.standard_normal((F, M, N)) + 1j * rng.standard_normal((F, M, N))
    G = rng.standard_normal((F, M, K, L)) + 1j * rng.standard_normal((F, M, K, L))
    p = rng.standard_normal(N)
    lhs = np.sum(np.conj(G) * O.estimate_real_pilot(Y, p, K, L)).real
    dY, _ = O.adjoint(G, Y, p, K, L)
    assert abs(lhs - np.sum(np.conj(dY) * Y).real) <= 1e-12 * abs(lhs)


# ------------------------------------------------------------------ quantisers


def _edge_values():
    rng = np.random.default_rng(0)
    v = np.concatenate([
        rng.standard_normal(20000) * 100.0,
        rng.standard_normal(20000) * 1e-3,
        np.ldexp(1.0 + np.arange(0, 64) / 64.0, -20),
        np.array([0.0, 1.0, -1.0, 1.5, 3.0, 0.1, 1e-8, 2.0 ** -24, 2.0 ** -25, 2.0 ** -26]),
    ])
    return v.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("fmt,tdt", [("fp16", "float16"), ("bf16", "bfloat16")])
def test_round_matches_torch_cast(fmt, tdt):
    torch = pytest.importorskip("torch")
    v = _edge_values()
    want = torch.tensor(v, dtype=torch.float32).to(getattr(torch, tdt)).double().numpy()
    assert np.array_equal(O.round_to_format(v, fmt), want)


@pytest.mark.parametrize("fmt,tdt", [("fp16", "float16"), ("bf16", "bfloat16")])
def test_round_overflow_and_non_finite_match_torch_cast(fmt, tdt):
    # IEEE 754 round to nearest past the largest finite value: the first magnitude that
    # rounds up out of the top binade becomes infinity; infinities and NaN pass through
    torch = pytest.importorskip("torch")
    vmax = O.FORMATS[fmt][2]
    mbits = O.FORMATS[fmt][0]
    half_ulp = np.ldexp(1.0, int(np.frexp(vmax)[1]) - 1 - mbits - 1)
    v = np.array([vmax, vmax + half_ulp, np.nextafter(np.float32(vmax + half_ulp), np.float32(0)),
                  1e30, np.float32(3.0e38), np.inf, -np.inf, -1e30, np.nan],
                 dtype=np.float32).astype(np.float64)
    want = torch.tensor(v, dtype=torch.float32).to(getattr(torch, tdt)).double().numpy()
    got = O.round_to_format(v, fmt)
    assert np.array_equal(got, want, equal_nan=True)
    assert got[1] == np.inf and got[2] == vmax     # the tie at the top rounds to even: up


def test_round_non_finite_hand_cases():
    # e4m3 has no infinity: overflow and infinite inputs saturate at +-448 (satfinite);
    # tf32 keeps float32's exponent range, so infinities stay infinite
    got = O.round_to_format([np.inf, -np.inf, np.nan, 1e6, -464.0, 463.0], "e4m3")
    assert got[0] == 448.0 and got[1] == -448.0 and np.isnan(got[2])
    assert list(got[3:]) == [448.0, -448.0, 448.0]
    got = O.round_to_format([np.inf, -np.inf, np.nan, 0.0], "tf32")
    assert got[0] == np.inf and got[1] == -np.inf and np.isnan(got[2]) and got[3] == 0.0
    # the largest tf32 value, and a float32 value that rounds (ties away) past it
    tmax = O.FORMATS["tf32"][2]
    assert O.round_to_format([tmax], "tf32")[0] == tmax
    assert O.round_to_format([np.ldexp(4095.0 / 2048.0, 127)], "tf32")[0] == np.inf


def test_quantize_assembles_parts_separately():
    # an infinite imaginary part must not leak into the real part of the operand
    Y = np.array([[[complex(1.0, np.inf), complex(np.nan, 0.5), 0.25 + 0j]]], np.complex64)
    Q, se = O.quantize(Y, "fp16")
    assert se[0, 0] == 0                                  # peak not finite: scale 1
    assert Q.real[0, 0, 0] == 1.0 and Q.imag[0, 0, 0] == np.inf
    assert np.isnan(Q.real[0, 0, 1]) and Q.imag[0, 0, 1] == 0.5
    D = O.dequantize(Q, se)
    assert D.real[0, 0, 0] == 1.0 and D.imag[0, 0, 0] == np.inf


def test_round_e4m3_matches_torch_cast_in_range():
    torch = pytest.importorskip("torch")
    v = _edge_values()
    v = v[np.abs(v) <= 448.0]
    want = torch.tensor(v, dtype=torch.float32).to(torch.float8_e4m3fn).double().numpy()
    assert np.array_equal(O.round_to_format(v, "e4m3"), want)


def test_round_tie_cases():
    one_half_ulp10 = 1.0 + 2.0 ** -11
    assert O.round_to_format([one_half_ulp10], "fp16")[0] == 1.0            # tie -> even
    assert O.round_to_format([one_half_ulp10], "tf32")[0] == 1.0 + 2.0 ** -10  # tie -> away
    assert O.round_to_format([-one_half_ulp10], "tf32")[0] == -(1.0 + 2.0 ** -10)
    assert list(O.round_to_format([17.0, 19.0, 448.0, 500.0, 2.0 ** -9, 2.0 ** -11], "e4m3")) == \
        [16.0, 20.0, 448.0, 448.0, 2.0 ** -9, 0.0]
    assert O.round_to_format([1.0 + 2.0 ** -8], "bf16")[0] == 1.0
    assert O.round_to_format([1.0 + 3 * 2.0 ** -8], "bf16")[0] == 1.0 + 2.0 ** -6


def test_scale_exponents():
    Y = np.zeros((1, 4, 3), np.complex64)
    Y[0, 0] = [1.0, 0.5j, -0.25]
    Y[0, 1] = [0.75, 0, 0]
    Y[0, 2] = [-3j, 0, 0]
    se16 = O.antenna_scale_exponents(Y, "fp16")[0]
    se8 = O.antenna_scale_exponents(Y, "e4m3")[0]
    assert list(se16) == [14, 15, 13, 0]
    assert list(se8) == [7, 8, 6, 0]
    assert list(O.antenna_scale_exponents(Y, "bf16")[0]) == [0, 0, 0, 0]
    Q, se = O.quantize(Y, "e4m3")
    peak = np.maximum(np.abs(Q.real), np.abs(Q.imag)).max(axis=-1)[0]
    assert np.all(peak[:3] >= 128) and np.all(peak[:3] < 256)


def test_scale_exponents_of_non_finite_peaks():
    # reading of the paper's silence on bad samples: a peak that is 0 or not finite gives
    # scale 1; a NaN part is left out of the peak
    Y = np.zeros((1, 4, 3), np.complex64)
    Y[0, 0] = [1.0, np.inf, 0.5]                     # infinite peak -> scale 1
    Y[0, 1] = [np.nan, 0.75, -0.25j]                  # NaN left out: peak 0.75
    Y[0, 2] = [complex(np.nan, np.nan)] * 3           # no number at all -> scale 1
    Y[0, 3] = [complex(0.0, -np.inf), 0, 0]
    for fmt, t in (("fp16", 15), ("e4m3", 8)):
        se = O.antenna_scale_exponents(Y, fmt)[0]
        assert list(se) == [0, t, 0, 0]


def test_quantized_estimate_within_stated_tolerances():
    bits, _, Y = _small_case(10, 16, 4, 64, 2, seed=9, snr=10.0)
    ref = O.estimate(Y, bits, 4, 64)
    for fmt, tol in (("fp16", 2e-3), ("bf16", 2e-3), ("e4m3", 3e-2), ("tf32", 1e-6)):
        assert O.nmse(O.estimate_quantized(Y, bits, 4, 64, fmt), ref) < tol


# ---------------------------------------------------------------------- metrics


def test_mae_eq12():
    est = np.array([[[[1 + 1j, 0]]]])
    h = np.array([[[[1, 3 + 4j]]]])
    assert O.mae(est, h) == pytest.approx((1 + 5) / 2)
    assert O.nmse(h, h) == 0.0


def test_nmse_hand_cases():
    # est = [3, 0], ref = [1, 1]: errors 2 and -1, so sum|e|^2 = 5 over sum|ref|^2 = 2.
    # Unsquared terms would give 3/2 = 1.5, dividing by sum|est|^2 would give 5/9.
    assert O.nmse(np.array([3.0, 0.0]), np.array([1.0, 1.0])) == 2.5
    # complex entries: est = [1+2i, 3i], ref = [1, 4i] -> errors 2i and -i, sum|e|^2 = 5;
    # sum|ref|^2 = 1 + 16 = 17 (not |1 + 4i|^2 summed per part wrongly as 1 + 4).
    assert O.nmse(np.array([1 + 2j, 3j]), np.array([1.0, 4j])) == pytest.approx(5 / 17, abs=0)
    # the metric is not symmetric: swapping the arguments changes the denominator
    assert O.nmse(np.array([1.0, 1.0]), np.array([3.0, 0.0])) == pytest.approx(5 / 9, abs=1e-15)
    # scaling both by the same factor leaves it unchanged (a ratio of like powers)
    assert O.nmse(np.array([30.0, 0.0]), np.array([10.0, 10.0])) == 2.5
    # shape is irrelevant: the sums run over all entries of a launch
    e = np.array([[[[3.0]], [[0.0]]]])
    r = np.array([[[[1.0]], [[1.0]]]])
    assert O.nmse(e, r) == 2.5


# ------------------------------------------- cyclic prefix and shift rules (Sec. II)


@pytest.mark.parametrize("shift_rule", ["kl", "spread"])
@pytest.mark.parametrize("r,M,K,L,cp", [(7, 3, 2, 16, 16), (9, 2, 4, 20, 31), (6, 2, 3, 5, 8)])
def test_cp_linear_channel_closed_form(r, M, K, L, cp, shift_rule):
    # a LINEAR channel on the CP-prefixed pilot, CP dropped at the receiver, gives the
    # circular model exactly (Sec. II-A), so the noise-free estimate is h + (h - S)/N
    bits = S.mseq_bits(r, 2)
    N = bits.size
    rng = np.random.default_rng(r)
    h = C.channel(rng, 2, M, K, L)
    sh = (C.shifts_kl if shift_rule == "kl" else C.shifts_spread)(K, L, N)
    Y = C.received_with_cp(h, bits, 0.0, rng, cp, shifts=sh, noise=False)
    H = O.estimate_general(Y, bits, K, L, cp_len=cp, shifts=sh)
    x = h.reshape(2, M, K * L)
    want = (x + (x - x.sum(-1, keepdims=True)) / N).reshape(h.shape)
    assert np.abs(H - want).max() <= 1e-5 * np.abs(want).max()


def test_cp_removal_matches_circular_generator():
    bits = S.mseq_bits(8, 0)
    rng = np.random.default_rng(0)
    h = C.channel(rng, 1, 4, 3, 12)
    y_cp = C.received_with_cp(h, bits, 0.0, rng, 12, noise=False)
    y_circ = C.received(h, bits, 0.0, rng, noise=False)
    assert np.abs(y_cp[..., 12:] - y_circ).max() <= 1e-5
    # general estimator with cp 0 and k*L shifts is the plain estimator
    assert np.abs(O.estimate_general(y_circ, bits, 3, 12) - O.estimate(y_circ, bits, 3, 12)).max() <= 1e-12


def test_spread_shift_rule_eq8():
    # Eq. 8: shift of transmitter t = (N / N_batch) * (t mod N_batch), floored
    assert list(C.shifts_spread(4, 16, 1023)) == [0, 255, 510, 765]
    with pytest.raises(ValueError):
        O.estimate_general(np.zeros((1, 1, 7), np.complex64), np.zeros(7, np.uint8), 2, 4,
                           shifts=[0, 3])          # lags 0..3 and 3..6 overlap
