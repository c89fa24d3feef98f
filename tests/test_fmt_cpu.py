"""Host logic of the fast m-sequence transform yardstick (pnce_fmt_tables), without a GPU.

The tables must make the transform reproduce the estimator of Eq. 3: the windows s_n are a
bijection onto the nonzero r-bit vectors and bit[(n - j) mod N] = parity(u_j & s_n) for
every sample n and lag j (checked exhaustively for small r, on samples for large r).  A
numpy Walsh-Hadamard transform driven by the tables is compared with the FP64 oracle, and
non-m-sequences are rejected.
"""
import numpy as np
import pytest

from oracle import pn_oracle as O
from synth import mseq

pk = pytest.importorskip("paper_2206_05506_gb300")


@pytest.fixture(scope="module")
def tables():
    try:
        pk.lib()
    except RuntimeError as e:           # library not built: the export test reports it
        pytest.skip(str(e))
    return pk.fmt_tables


def _parity(x):
    x = x.astype(np.uint32)
    p = np.zeros_like(x)
    while np.any(x):
        p ^= x & 1
        x >>= 1
    return p


@pytest.mark.parametrize("r", [2, 3, 4, 5, 7, 8])
@pytest.mark.parametrize("seed", [0, 1])
def test_tables_exhaustive(tables, r, seed):
    bits = mseq.mseq_bits(r, seed)
    N = bits.size
    pos, lag = tables(bits)
    assert sorted(pos.tolist()) == list(range(1, N + 1))
    n = np.arange(N)
    for j in range(N):
        assert np.array_equal(_parity(lag[j] & pos.astype(np.uint32)), bits[(n - j) % N]), j


@pytest.mark.parametrize("r", [10, 12, 14])
def test_tables_sampled(tables, r):
    bits = mseq.mseq_bits(r, 3)
    N = bits.size
    pos, lag = tables(bits)
    assert np.array_equal(np.sort(pos), np.arange(1, N + 1))
    rng = np.random.default_rng(r)
    n = np.arange(N)
    for j in rng.choice(N, 16, replace=False):
        assert np.array_equal(_parity(lag[j] & pos.astype(np.uint32)), bits[(n - j) % N])


def _wht(x):
    """Walsh-Hadamard transform (unnormalised) along the last axis, length 2^r."""
    x = x.copy()
    h = 1
    S = x.shape[-1]
    while h < S:
        y = x.reshape(*x.shape[:-1], S // (2 * h), 2, h)
        a, b = y[..., 0, :].copy(), y[..., 1, :].copy()
        y[..., 0, :], y[..., 1, :] = a + b, a - b
        x = y.reshape(*x.shape[:-1], S)
        h *= 2
    return x


@pytest.mark.parametrize("r,K,L", [(3, 1, 7), (5, 3, 10), (9, 4, 100), (11, 8, 128)])
def test_table_driven_transform_equals_oracle(tables, r, K, L):
    bits = mseq.mseq_bits(r, 1)
    N = bits.size
    rng = np.random.default_rng(r)
    Y = rng.standard_normal((2, 3, N)) + 1j * rng.standard_normal((2, 3, N))
    pos, lag = tables(bits)
    X = np.zeros((2, 3, N + 1), dtype=complex)
    X[..., pos.astype(np.int64)] = Y
    W = _wht(X)
    H = (W[..., lag[: K * L].astype(np.int64)] / N).reshape(2, 3, K, L)
    ref = O.estimate(Y, bits, K, L)
    assert np.max(np.abs(H - ref)) < 1e-12


def test_rejects_non_msequences(tables):
    bits = mseq.mseq_bits(7, 0)
    bad = bits.copy()
    bad[5] ^= 1                                  # one flipped bit: no longer linear
    with pytest.raises(pk.PnceError):
        tables(bad)
    with pytest.raises(pk.PnceError):
        tables(np.random.default_rng(0).integers(0, 2, 127))
    with pytest.raises(pk.PnceError):
        tables(np.ones(100, dtype=np.uint8))       # N + 1 not a power of two
    with pytest.raises(pk.PnceError):
        tables(mseq.mseq_bits(15, 0))             # 2^15 entries exceed the transform's limit
