"""GPU parity of the fast m-sequence transform yardstick (pnce_estimate_fmt) against the
FP64 oracle: FP32 sums of +-y over r butterfly levels, NMSE <= 1e-10, on shapes from the
smallest degree to the precision workload's N = 4095, with ragged row counts, the
full-lag case K*L = N and K = L = 1; plus its agreement with the FP32 SIMT path and the
argument checks."""
import numpy as np
import pytest
import torch

from oracle import pn_oracle as O
from synth import channel as C

pytestmark = pytest.mark.gpu

# (r, M, K, L, F)
SHAPES = [(2, 1, 1, 3, 1), (3, 5, 1, 7, 2), (5, 3, 2, 9, 1), (7, 8, 2, 16, 3),
          (10, 37, 8, 64, 2), (12, 128, 16, 128, 2), (9, 2, 1, 1, 1), (13, 4, 2, 300, 1),
          (11, 3, 1, 2047, 1), (14, 2, 2, 100, 1)]


@pytest.fixture(scope="module")
def pk():
    import paper_2206_05506_gb300 as pk
    pk.lib()
    return pk


@pytest.mark.parametrize("shape", SHAPES)
def test_fmt_matches_oracle(pk, shape):
    r, M, K, L, F = shape
    w = C.Workload("t", r=r, M=M, K=K, L=L, F=F, snr_db=(10.0,), seed=r)
    bits, _, Y = C.make(w)
    dev = torch.device("cuda", 0)
    fmt = pk.FmtPilot(bits, device=dev)
    n = F * M * K * L
    buf = torch.full((n + 64,), complex(7.0, 7.0), dtype=torch.complex64, device=dev)
    H = buf[32:32 + n].view(F, M, K, L)
    pk.estimate_fmt(torch.from_numpy(Y).to(dev), fmt, K, L, out=H)
    assert pk.get_status(dev) == 0
    g = torch.cat([buf[:32], buf[-32:]]).cpu().numpy()
    assert np.all(g == np.complex64(complex(7.0, 7.0))), "write outside H"
    ref = O.estimate(Y, bits, K, L)
    assert O.nmse(H.cpu().numpy(), ref) <= 1e-10


def test_fmt_agrees_with_simt(pk):
    w = C.Workload("t", r=11, M=64, K=8, L=64, F=4, snr_db=(0.0,), seed=5)
    bits, _, Y = C.make(w)
    dev = torch.device("cuda", 0)
    Yd = torch.from_numpy(Y).to(dev)
    a = pk.estimate_fmt(Yd, pk.FmtPilot(bits, device=dev), 8, 64).cpu().numpy()
    b = pk.estimate(Yd, pk.Pilot(bits, device=dev), 8, 64, dtype="fp32").cpu().numpy()
    assert O.nmse(a, b) <= 1e-10


def test_fmt_rejects_bad_arguments(pk):
    dev = torch.device("cuda", 0)
    w = C.Workload("t", r=7, M=2, K=2, L=16, F=1, snr_db=(10.0,), seed=0)
    bits, _, Y = C.make(w)
    fmt = pk.FmtPilot(bits, device=dev)
    Yd = torch.from_numpy(Y).to(dev)
    with pytest.raises(pk.PnceError):
        pk.estimate_fmt(Yd, fmt, 16, 16)                 # K*L > N
    with pytest.raises(ValueError):
        pk.estimate_fmt(Yd[..., :100].contiguous(), fmt, 2, 16)   # N mismatch
    with pytest.raises(pk.PnceError):
        pk.FmtPilot(np.ones(127, dtype=np.uint8), device=dev)    # not an m-sequence
