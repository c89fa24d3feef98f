"""Parity at the full precision workload (512 frames x 128 antennas, N = 4095, K = 16,
L = 128), in the launch configuration the benchmark times (pnce_estimate: quantise, then
correlate), and with the optional chunked overlap of the two.  The oracle checks sampled
frames one by one; per-antenna scales are checked for every antenna."""
import numpy as np
import pytest
import torch

from oracle import pn_oracle as O
from synth import channel as C

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-6, "tf32": 1e-6, "fp16": 2e-3, "bf16": 2e-3, "e4m3": 3e-2}
TOL_Q = {"tf32": 1e-9, "fp16": 1e-9, "bf16": 1e-9, "e4m3": 1e-6}
SAMPLE = [0, 1, 257, 510, 511]


@pytest.fixture(scope="module")
def full():
    import paper_2206_05506_gb300 as pk
    w = C.PRECISION
    bits, Y = C.make_received(w)
    dev = torch.device("cuda", 0)
    Yd = torch.from_numpy(Y).to(dev)
    pilot = pk.Pilot(bits, device=dev)
    return pk, w, bits, Y, Yd, pilot


@pytest.mark.parametrize("dtype", ["fp16", "e4m3", "bf16", "tf32", "fp32"])
def test_full_size_sampled_frames(full, dtype):
    pk, w, bits, Y, Yd, pilot = full
    H = pk.estimate(Yd, pilot, w.K, w.L, dtype=dtype)
    assert pk.get_status(Yd.device) == 0
    Hs = H[SAMPLE].cpu().numpy()
    Ys = Y[SAMPLE]
    ref = O.estimate(Ys, bits, w.K, w.L)
    assert O.nmse(Hs, ref) <= TOL[dtype]
    if dtype != "fp32":
        assert O.nmse(Hs, O.estimate_quantized(Ys, bits, w.K, w.L, dtype)) <= TOL_Q[dtype]
    # every frame is finite and of the expected size (taps have unit power per link)
    p = H.abs().pow(2).sum(dim=(2, 3)).mean().item()
    assert np.isfinite(p) and 0.5 * w.K < p < 2.0 * w.K


@pytest.mark.parametrize("chunks", ["2", "4", "8"])
@pytest.mark.parametrize("dtype", ["fp16", "e4m3"])
def test_overlapped_equals_sequential(full, dtype, chunks, monkeypatch):
    # the chunked, overlapped pnce_estimate gives the same bits as quantise-then-correlate
    pk, w, bits, Y, Yd, pilot = full
    monkeypatch.setenv("PNCE_OVERLAP_CHUNKS", chunks)
    H = pk.estimate(Yd, pilot, w.K, w.L, dtype=dtype)
    monkeypatch.delenv("PNCE_OVERLAP_CHUNKS")
    q = pk.quantize(Yd, dtype)
    H2 = pk.correlate_quantized(q["workspace"], pilot, w.F, w.M, w.K, w.L, dtype)
    assert torch.equal(H, H2)


def test_full_size_scales_every_antenna(full):
    pk, w, bits, Y, Yd, pilot = full
    for dtype in ("fp16", "e4m3"):
        q = pk.quantize(Yd, dtype)
        want = O.antenna_scale_exponents(Y, dtype).reshape(-1)
        assert np.array_equal(q["exps"].cpu().numpy(), want)
