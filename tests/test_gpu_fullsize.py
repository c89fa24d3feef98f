"""Parity at the full precision workload (512 frames x 128 antennas, N = 4095, K = 16,
L = 128), in the launch configuration the benchmark times (pnce_estimate: quantise, then
correlate), and with the optional chunked overlap of the two.

Every frame of every dtype is compared with the oracle: against the FP64 estimate of the
complex64 input (the stated accuracy targets, also per SNR of the sweep) and, for the
tensor-core dtypes, against the FP64 estimate of the quantised operand (which isolates the
FP32 accumulation), per frame.  The oracle runs in spawned worker processes, one chunk
of frames each (tests/fullsize_oracle.py); per-antenna scales are checked for every
antenna."""
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest
import torch

from oracle import pn_oracle as O
from synth import channel as C

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-6, "tf32": 1e-6, "fp16": 2e-3, "bf16": 2e-3, "e4m3": 3e-2}
TOL_Q = {"tf32": 1e-9, "fp16": 1e-9, "bf16": 1e-9, "e4m3": 1e-6}
DTYPES = ["fp16", "e4m3", "bf16", "tf32", "fp32"]
CHUNK = 16


@pytest.fixture(scope="module")
def full():
    import paper_2206_05506_gb300 as pk
    w = C.PRECISION
    bits, Y = C.make_received(w)
    dev = torch.device("cuda", 0)
    Yd = torch.from_numpy(Y).to(dev)
    pilot = pk.Pilot(bits, device=dev)
    return pk, w, bits, Y, Yd, pilot


@pytest.fixture(scope="module")
def all_frames(full):
    """GPU estimates of all 512 frames for every dtype, and the oracle's per-frame sums."""
    pk, w, bits, Y, Yd, pilot = full
    gpu = {}
    for dtype in DTYPES:
        H = pk.estimate(Yd, pilot, w.K, w.L, dtype=dtype)
        assert pk.get_status(Yd.device) == 0
        gpu[dtype] = H.cpu().numpy()
        del H
    torch.cuda.empty_cache()
    workers = max(1, min(16, len(os.sched_getaffinity(0))))
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")   # one BLAS thread each
    try:
        import fullsize_oracle as FO
        with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            futs = [ex.submit(FO.chunk_stats, f0, CHUNK,
                              {d: gpu[d][f0:f0 + CHUNK] for d in DTYPES})
                    for f0 in range(0, w.F, CHUNK)]
            parts = [f.result() for f in futs]
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    stats = {d: tuple(np.concatenate([p[d][i] for p in parts]) for i in range(4)) for d in DTYPES}
    stats["fp32_maxabs"] = max(p["fp32_maxabs"] for p in parts)
    return w, gpu, stats


@pytest.mark.parametrize("dtype", DTYPES)
def test_full_size_every_frame(all_frames, dtype):
    w, gpu, stats = all_frames
    num, numq, den, denq = stats[dtype]
    assert num.shape == (w.F,) and np.all(den > 0)
    assert num.sum() / den.sum() <= TOL[dtype]                  # the launch
    assert np.max(num / den) <= TOL[dtype]                      # every frame
    snr = w.frame_snr()
    for s in np.unique(snr):                                    # every SNR of the sweep
        f = snr == s
        assert num[f].sum() / den[f].sum() <= TOL[dtype], s
    if dtype == "fp32":
        assert stats["fp32_maxabs"] <= 1e-5
    else:
        assert numq.sum() / denq.sum() <= TOL_Q[dtype]
        assert np.max(numq / denq) <= TOL_Q[dtype]


def test_full_size_every_frame_finite(all_frames):
    w, gpu, stats = all_frames
    for dtype in DTYPES:
        H = gpu[dtype]
        assert np.isfinite(H.view(np.float32)).all(), dtype
        p = (np.abs(H) ** 2).sum(axis=(2, 3)).mean()
        assert 0.5 * w.K < p < 2.0 * w.K


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
