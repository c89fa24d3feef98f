"""Seeded random shapes through every arithmetic and both pilot-slot layouts, against the
FP64 oracle: sequence degrees 2..12, ragged antenna counts (1..70, so the 8-antenna groups
and 128-row tiles are partly filled), lag counts from 1 to N, cyclic prefixes, the spread
shift rule.  Tolerances as in test_gpu_parity (NMSE against the oracle on the quantised
operand for the tensor-core formats, against the unquantised input for FP32)."""
import numpy as np
import pytest
import torch

from oracle import pn_oracle as O
from synth import channel as C
from synth import mseq

pytestmark = pytest.mark.gpu

TOL_Q = {"tf32": 1e-9, "fp16": 1e-9, "bf16": 1e-9, "e4m3": 1e-6}


def _cases(n=40, seed=2024):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        r = int(rng.integers(2, 13))
        N = (1 << r) - 1
        rule = "spread" if rng.random() < 0.3 else "kl"
        K = int(rng.integers(1, min(N, 16) + 1))
        Lmax = N // K
        L = int(rng.integers(1, Lmax + 1))
        M = int(rng.integers(1, 71))
        F = int(rng.integers(1, 4))
        cp = int(rng.integers(0, min(L, 40) + 1)) if rng.random() < 0.4 else 0
        dtype = ["fp32", "fp16", "bf16", "e4m3", "tf32"][i % 5]
        out.append((r, M, K, L, F, cp, rule, dtype, i))
    return out


@pytest.fixture(scope="module")
def pk():
    import paper_2206_05506_gb300 as pk
    pk.lib()
    return pk


@pytest.mark.parametrize("case", _cases())
def test_random_shape_matches_oracle(pk, case):
    r, M, K, L, F, cp, rule, dtype, i = case
    bits = mseq.mseq_bits(r, i % 3)
    N = bits.size
    rng = np.random.default_rng([7, i])
    h = C.channel(rng, F, M, K, L)
    sh = (C.shifts_kl if rule == "kl" else C.shifts_spread)(K, L, N)
    Y = C.received_with_cp(h, bits, 10.0, rng, cp, shifts=sh)
    dev = torch.device("cuda", 0)
    pilot = pk.Pilot(bits, device=dev)
    n = F * M * K * L
    buf = torch.full((n + 64,), complex(4.0, 4.0), dtype=torch.complex64, device=dev)
    H = buf[32:32 + n].view(F, M, K, L)
    pk.estimate(torch.from_numpy(Y).to(dev), pilot, K, L, dtype=dtype, out=H, cp_len=cp,
                shift_rule=rule)
    assert pk.get_status(dev) == 0
    g = torch.cat([buf[:32], buf[-32:]]).cpu().numpy()
    assert np.all(g == np.complex64(complex(4.0, 4.0))), "write outside H"
    got = H.cpu().numpy()
    if dtype == "fp32":
        ref = O.estimate_general(Y, bits, K, L, cp_len=cp, shifts=sh)
        assert O.nmse(got, ref) <= 1e-6
    else:
        Yc = np.ascontiguousarray(Y[..., cp:])
        ref = O.estimate_general(O.dequantize(*O.quantize(Yc, dtype)), bits, K, L, cp_len=0,
                                 shifts=sh)
        assert O.nmse(got, ref) <= TOL_Q[dtype]
