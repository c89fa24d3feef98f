"""FP64 CPU oracle for PN-sequence correlation channel estimation.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or link this
module: only the tests, the smoke check in __graft_entry__, and bench.py's CPU-baseline
leg and its reference arm use it.  It shares no code with the CUDA library.

Everything is plain numpy in float64 (complex128), written from the paper's
definitions so that it can be checked by eye:

* pilot symbols: the PN bits are BPSK-mapped, bit 0 -> +1 and bit 1 -> -1 (the
  paper fixes only that the pilot is a real +-1 PN sequence, Sec. II-A; the sign
  convention cancels because the same pilot is used to transmit and to correlate);
* circulant pilot matrix, Eq. 2: S[i, j] = s[(i - j) mod N] (first row
  [s_0, s_{N-1}, ..., s_1]);
* correlation estimator, Eq. 3 / Eq. 10: H_hat = (1/N) S^T Y, i.e. for every antenna
  row y, H_hat[j] = (1/N) sum_n y[n] s[(n - j) mod N], kept for lags j < K*L.  With
  transmitter k multiplexed by the cyclic shift k*L (Sec. II-B, Eq. 8 with the shift
  k*L), lag j = k*L + l is tap l of transmitter k.

Three independent forms of that definition are provided: a brute-force loop
(`estimate_direct`, tiny inputs), the explicit Toeplitz product (`estimate`, the
timed CPU baseline) and an FFT circular correlation (`estimate_fft`).

Also here: the adjoint of the estimator with respect to the received block and to a
real-valued relaxed pilot, the quantisers that define the reduced-precision operand
(round-to-nearest onto the fp16 / bf16 / fp8-e4m3 / tf32 grids with a per-antenna
power-of-two scale), and the NMSE / MAE metrics (MAE is Eq. 12).
"""
from __future__ import annotations

import numpy as np

# --------------------------------------------------------------------------- pilot


def pilot_symbols(bits) -> np.ndarray:
    """BPSK pilot: bit 0 -> +1.0, bit 1 -> -1.0 (float64)."""
    b = np.asarray(bits).astype(np.int64)
    if np.any((b != 0) & (b != 1)):
        raise ValueError("pilot bits must be 0/1")
    return np.where(b == 0, 1.0, -1.0)


def pilot_matrix(p: np.ndarray, ncols: int) -> np.ndarray:
    """First `ncols` columns of the N x N circulant of Eq. 2: P[n, j] = p[(n - j) mod N]."""
    p = np.asarray(p, dtype=np.float64)
    N = p.size
    n = np.arange(N)[:, None]
    j = np.arange(ncols)[None, :]
    return p[(n - j) % N]


def _check_shape(Y, K, L):
    if Y.ndim != 3:
        raise ValueError("Y must be [F, M, N]")
    N = Y.shape[-1]
    if K < 1 or L < 1 or K * L > N:
        raise ValueError("need K, L >= 1 and K*L <= N (Eq. 7 with C = L)")
    return N


# ------------------------------------------------------------------- estimators


def estimate_direct(Y, bits, K: int, L: int) -> np.ndarray:
    """O1: brute-force H_hat[f,m,k,l] = (1/N) sum_n y[f,m,n] p[(n - l - kL) mod N]."""
    Y = np.asarray(Y).astype(np.complex128)
    N = _check_shape(Y, K, L)
    p = pilot_symbols(bits)
    F, M, _ = Y.shape
    H = np.zeros((F, M, K, L), dtype=np.complex128)
    for f in range(F):
        for m in range(M):
            for k in range(K):
                for l in range(L):
                    acc = 0j
                    for n in range(N):
                        acc += Y[f, m, n] * p[(n - l - k * L) % N]
                    H[f, m, k, l] = acc / N
    return H


def estimate_real_pilot(Y, p, K: int, L: int, chunk_rows: int = 4096) -> np.ndarray:
    """O2 with an arbitrary real pilot p: H_hat = (1/N) Y P, P = pilot_matrix(p, K*L).

    The complex product is taken as two real products (real and imaginary parts of Y),
    in float64 through numpy's BLAS, chunked over antenna rows.
    """
    Y = np.asarray(Y)
    N = _check_shape(Y, K, L)
    F, M, _ = Y.shape
    P = pilot_matrix(p, K * L)
    rows = Y.reshape(F * M, N)
    out = np.empty((F * M, K * L), dtype=np.complex128)
    for r0 in range(0, F * M, chunk_rows):
        blk = rows[r0:r0 + chunk_rows]
        re = blk.real.astype(np.float64) @ P
        im = blk.imag.astype(np.float64) @ P
        out[r0:r0 + chunk_rows] = (re + 1j * im) / N
    return out.reshape(F, M, K, L)


def estimate(Y, bits, K: int, L: int) -> np.ndarray:
    """O2: the explicit Toeplitz form of Eq. 3 / Eq. 10 with the BPSK pilot."""
    return estimate_real_pilot(Y, pilot_symbols(bits), K, L)


def estimate_general(Y, bits, K: int, L: int, cp_len: int = 0, shifts=None) -> np.ndarray:
    """Estimator for rows that still carry a cyclic prefix and/or other cyclic shifts.

    Y[f, m, cp_len + n] holds received sample n after the prefix (Sec. II-A: the CP is
    removed before correlating); transmitter k uses the cyclic shift shifts[k] (default
    k*L; Eq. 8 spreads them evenly).  H_hat[f,m,k,l] = (1/N) sum_n y[n] p[(n - shifts[k] - l)
    mod N]: the correlator of Eq. 3 evaluated at the lags shifts[k] + l.
    """
    Y = np.asarray(Y)
    if Y.ndim != 3:
        raise ValueError("Y must be [F, M, cp_len + N]")
    p = pilot_symbols(bits)
    N = p.size
    if Y.shape[-1] != cp_len + N:
        raise ValueError("rows must hold cp_len + N samples")
    sh = np.arange(K) * L if shifts is None else np.asarray(shifts, dtype=np.int64)
    lags = (sh[:, None] + np.arange(L)[None, :]).reshape(-1)
    if np.unique(lags % N).size != lags.size:
        raise ValueError("the lag sets of different transmitters overlap (aliasing)")
    y = Y[..., cp_len:].astype(np.complex128)
    F, M, _ = y.shape
    P = p[(np.arange(N)[:, None] - lags[None, :]) % N]
    rows = y.reshape(F * M, N)
    H = (rows.real @ P + 1j * (rows.imag @ P)) / N
    return H.reshape(F, M, K, L)


def estimate_fft(Y, bits, K: int, L: int) -> np.ndarray:
    """O3: circular cross-correlation by DFT, ifft(fft(y) * conj(fft(p))) / N, lags < K*L."""
    Y = np.asarray(Y).astype(np.complex128)
    N = _check_shape(Y, K, L)
    F, M, _ = Y.shape
    p = pilot_symbols(bits)
    c = np.fft.ifft(np.fft.fft(Y, axis=-1) * np.conj(np.fft.fft(p)), axis=-1) / N
    return c[..., : K * L].reshape(F, M, K, L)


# ---------------------------------------------------------------------- adjoint


def adjoint(G, Y, p, K: int, L: int):
    """Gradients of a real loss through H_hat = (1/N) Y P(p), P[n,j] = p[(n-j) mod N].

    G[f,m,k,l] is dLoss/dRe(H_hat) + i dLoss/dIm(H_hat) (PyTorch's convention for
    complex tensors).  Returns
      dY[f,m,n] = (1/N) sum_j G[f,m,j] p[(n - j) mod N]            (= G P^T / N)
      dp[q]     = (1/N) sum_{f,m,j} Re(conj(G[f,m,j]) Y[f,m,(q + j) mod N])
    from the chain rule on the linear map (dH_hat[.,j]/dp[q] = Y[., (q+j) mod N] / N).
    """
    Y = np.asarray(Y).astype(np.complex128)
    N = _check_shape(Y, K, L)
    F, M, _ = Y.shape
    p = np.asarray(p, dtype=np.float64)
    Gm = np.asarray(G).astype(np.complex128).reshape(F * M, K * L)
    P = pilot_matrix(p, K * L)
    dY = (Gm.real @ P.T + 1j * (Gm.imag @ P.T)) / N
    rows = Y.reshape(F * M, N)
    dp = np.zeros(N, dtype=np.float64)
    for j in range(K * L):
        shifted = np.roll(rows, -j, axis=1)        # shifted[:, q] = Y[:, (q + j) mod N]
        dp += (Gm[:, j].real[:, None] * shifted.real
               + Gm[:, j].imag[:, None] * shifted.imag).sum(axis=0)
    return dY.reshape(F, M, N), dp / N


# ---------------------------------------------------------------- quantisation

# (mantissa bits, minimum normal exponent, largest finite value, ties)
FORMATS = {
    "fp16": (10, -14, 65504.0, "even"),
    "bf16": (7, -126, float(np.ldexp(255.0 / 128.0, 127)), "even"),
    "tf32": (10, -126, float(np.ldexp(2047.0 / 1024.0, 127)), "away"),
    "e4m3": (3, -6, 448.0, "even"),
}

# exponent target: the per-antenna peak component is scaled into [2^(t-1), 2^t)
SCALE_TARGET_EXP = {"fp16": 15, "e4m3": 8, "bf16": None, "tf32": None, "fp32": None}


def round_to_format(x, fmt: str) -> np.ndarray:
    """Round float64 values to the nearest value of a binary format, by definition.

    The grid spacing at |x| is 2^(max(e, emin) - mbits) with e = floor(log2|x|); values
    are rounded to that grid (ties to even, or away from zero for tf32).  A rounded
    magnitude above the largest finite value overflows as IEEE 754 rounding to nearest
    prescribes: to infinity for the formats that have one (fp16, bf16, tf32); e4m3 has
    no infinity and saturates at 448 instead (the satfinite convention).  Infinite inputs
    follow the same rule (inf for fp16 / bf16 / tf32, +-448 for e4m3); NaN stays NaN.
    """
    mbits, emin, vmax, ties = FORMATS[fmt]
    x = np.asarray(x, dtype=np.float64)
    top = vmax if fmt == "e4m3" else np.inf     # where an overflowing magnitude lands
    out = np.full(x.shape, np.nan)              # NaN stays NaN
    inf = np.isinf(x)
    out[inf] = np.sign(x[inf]) * top
    fin = np.isfinite(x)
    out[fin & (x == 0)] = 0.0
    nz = fin & (x != 0)
    ax = np.abs(x[nz])
    _, E = np.frexp(ax)                         # ax = m 2^E, m in [0.5, 1)
    e = np.maximum(E - 1, emin)
    ulp = np.ldexp(1.0, e - mbits)
    q = ax / ulp                                # exact: division by a power of two
    if ties == "even":
        rq = np.rint(q)                         # round half to even
    else:
        rq = np.floor(q + 0.5)                  # round half away from zero
    v = rq * ulp
    v = np.where(v > vmax, top, v)
    out[nz] = np.sign(x[nz]) * v
    return out


def antenna_scale_exponents(Y, fmt: str) -> np.ndarray:
    """Per-antenna power-of-two scale exponent s_e (scale = 2^s_e), int32 [F, M].

    A = max_n max(|Re y[n]|, |Im y[n]|) over the parts that are numbers (a NaN part is
    left out of the peak); for fp16 / e4m3, s_e = t - E where A = m 2^E, m in [0.5, 1),
    so that the scaled peak lies in [2^(t-1), 2^t); for bf16, tf32 and fp32, and for a
    peak that is 0 or not finite (an infinite part, or no number at all), s_e = 0, i.e.
    scale 1.  s_e is clamped to [-100, 100].
    """
    Y = np.asarray(Y)
    t = SCALE_TARGET_EXP[fmt]
    F, M, _ = Y.shape
    if t is None:
        return np.zeros((F, M), dtype=np.int32)
    parts = np.fmax(np.abs(Y.real), np.abs(Y.imag)).astype(np.float64)   # fmax skips NaN
    A = np.fmax.reduce(parts, axis=-1)
    ok = np.isfinite(A) & (A > 0)
    _, E = np.frexp(np.where(ok, A, 1.0))
    se = np.where(ok, t - E, 0)
    return np.clip(se, -100, 100).astype(np.int32)


def quantize(Y, fmt: str):
    """The reduced-precision operand the tensor cores consume.

    Returns (Q, se): Q[f,m,n] = round(y * 2^se) in `fmt` (complex128 holding the
    rounded real and imaginary parts), se the per-antenna exponent.
    """
    Y = np.asarray(Y)
    se = antenna_scale_exponents(Y, fmt)
    s = np.ldexp(1.0, se)[..., None]
    Q = np.empty(Y.shape, dtype=np.complex128)
    # assembled part by part: re + 1j * im would turn an infinite imaginary part into a
    # NaN real part (1j * inf = nan + inf j in complex arithmetic)
    Q.real = round_to_format(Y.real.astype(np.float64) * s, fmt)
    Q.imag = round_to_format(Y.imag.astype(np.float64) * s, fmt)
    return Q, se


def dequantize(Q, se) -> np.ndarray:
    """Undo the exact per-antenna scale, part by part (see quantize)."""
    s = np.ldexp(1.0, -np.asarray(se))[..., None]
    out = np.empty(np.broadcast_shapes(Q.shape, s.shape), dtype=np.complex128)
    out.real = Q.real * s
    out.imag = Q.imag * s
    return out


def estimate_quantized(Y, bits, K: int, L: int, fmt: str) -> np.ndarray:
    """Estimator applied, in float64, to the quantised operand (undoing the exact scale)."""
    Q, se = quantize(Y, fmt)
    return estimate(dequantize(Q, se), bits, K, L)


# ---------------------------------------------------------------------- metrics


def nmse(est, ref) -> float:
    """sum |est - ref|^2 / sum |ref|^2 over all entries."""
    est = np.asarray(est).astype(np.complex128)
    ref = np.asarray(ref).astype(np.complex128)
    den = np.sum(np.abs(ref) ** 2)
    return float(np.sum(np.abs(est - ref) ** 2) / den) if den > 0 else float(np.sum(np.abs(est) ** 2))


def mae(est, h_true) -> float:
    """Eq. 12: mean over (transmitter, receiver, tap) of |h_hat - h|."""
    return float(np.mean(np.abs(np.asarray(est) - np.asarray(h_true))))
