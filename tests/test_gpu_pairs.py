"""GPU parity of the 2-SM tensor-core variant (CTA pairs, PNCE_TC_PAIRS=1) against the oracle.

The pair kernel computes 256-row tiles with tcgen05.mma.cta_group::2, each CTA of the pair
holding half of the tile's pilot list.  The bar is the one of the 1-CTA kernel: within FP32
accumulation of the quantised operand (NMSE <= 1e-9, 1e-6 for e4m3), on shapes with one and
several lag blocks, ragged row and lag tiles, the spread shift rule and a CP, plus the
full-size lag width with several pair tiles per pair.
"""
import numpy as np
import pytest
import torch

from oracle import pn_oracle as O
from synth import channel as C

pytestmark = pytest.mark.gpu

TOL_Q = {"tf32": 1e-9, "fp16": 1e-9, "bf16": 1e-9, "e4m3": 1e-6}
TC = ["fp16", "bf16", "e4m3", "tf32"]
GUARD = 64
SENT = complex(12345.0, -777.0)

# (r, M, K, L, F): one lag block and one pair tile; ragged rows (odd CTA idle); two lag
# blocks with ragged lags; eight lag blocks of 256 lags; many pair tiles per pair
SHAPES = [(7, 8, 2, 16, 1), (6, 3, 7, 9, 2), (10, 100, 5, 60, 3), (12, 64, 16, 128, 2),
          (11, 200, 4, 100, 9)]


@pytest.fixture(scope="module")
def pk():
    import paper_2206_05506_gb300 as pk
    pk.lib()
    return pk


@pytest.fixture
def pairs(monkeypatch):
    monkeypatch.setenv("PNCE_TC_PAIRS", "1")


def _run(pk, Y, bits, K, L, dtype, **kw):
    dev = torch.device("cuda", 0)
    pilot = pk.Pilot(bits, device=dev)
    F, M, N = Y.shape
    n = F * M * K * L
    buf = torch.full((n + 2 * GUARD,), SENT, dtype=torch.complex64, device=dev)
    H = buf[GUARD:GUARD + n].view(F, M, K, L)
    pk.estimate(torch.from_numpy(Y).to(dev), pilot, K, L, dtype=dtype, out=H, **kw)
    assert pk.get_status(dev) == 0
    g = torch.cat([buf[:GUARD], buf[-GUARD:]]).cpu().numpy()
    assert np.all(g == np.complex64(SENT)), "write outside H"
    return H.cpu().numpy()


@pytest.mark.parametrize("dtype", TC)
@pytest.mark.parametrize("shape", SHAPES)
def test_pair_kernel_matches_oracle(pk, pairs, shape, dtype):
    r, M, K, L, F = shape
    w = C.Workload("t", r=r, M=M, K=K, L=L, F=F, snr_db=(10.0,), seed=r + 3)
    bits, _, Y = C.make(w)
    H = _run(pk, Y, bits, K, L, dtype)
    refq = O.estimate_quantized(Y, bits, K, L, dtype)
    assert O.nmse(H, refq) <= TOL_Q[dtype]


@pytest.mark.parametrize("dtype", ["fp16", "e4m3"])
def test_pair_kernel_spread_shifts_and_cp(pk, pairs, dtype):
    rng = np.random.default_rng(7)
    N, K, L, cp = 1023, 4, 70, 40
    bits = (rng.random(N) < 0.5).astype(np.uint8)
    Y = (rng.standard_normal((2, 50, N + cp)) + 1j * rng.standard_normal((2, 50, N + cp)))
    Y = Y.astype(np.complex64)
    H = _run(pk, Y, bits, K, L, dtype, cp_len=cp, shift_rule="spread")
    shifts = C.shifts_spread(K, L, N)
    Yq = O.dequantize(*O.quantize(np.ascontiguousarray(Y[..., cp:]), dtype))
    ref = O.estimate_general(Yq, bits, K, L, cp_len=0, shifts=shifts)
    assert O.nmse(H, ref) <= TOL_Q[dtype]


def test_pair_kernel_equals_single_cta_kernel(pk, monkeypatch):
    # same operand, same FP32 accumulation: the two variants agree to rounding order
    w = C.Workload("t", r=12, M=128, K=16, L=128, F=16, snr_db=(10.0,), seed=1)
    bits, _, Y = C.make(w)
    base = _run(pk, Y, bits, 16, 128, "fp16")
    monkeypatch.setenv("PNCE_TC_PAIRS", "1")
    pair = _run(pk, Y, bits, 16, 128, "fp16")
    assert O.nmse(pair, base) <= 1e-12
