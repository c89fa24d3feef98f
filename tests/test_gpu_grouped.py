"""pnce_estimate_grouped (serving batches) against per-request pnce_estimate: requests of
uneven M, K, L sharing one pilot, buffers in device and in page-locked host memory, empty
slots, an invalid descriptor (skipped, status latched, the others unaffected) and replays
of a captured graph with rewritten descriptors."""
import ctypes as C

import numpy as np
import pytest
import torch

from synth import channel as C_
from synth import mseq

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    import paper_2206_05506_gb300 as pk
    pk.lib()
    return pk


def _table(pk, n):
    from paper_2206_05506_gb300 import _lib
    buf = torch.zeros(n * C.sizeof(_lib.ReqDesc), dtype=torch.uint8, pin_memory=True)
    arr = (_lib.ReqDesc * n).from_address(buf.data_ptr())
    return buf, arr


def _requests(N, specs, seed, host):
    rng = np.random.default_rng(seed)
    out = []
    for M, K, L in specs:
        Y = (rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))).astype(np.complex64)
        Yt = torch.from_numpy(Y)
        Yt = Yt.pin_memory() if host else Yt.cuda()
        Ht = torch.full((M, K * L), complex(5.0, 5.0), dtype=torch.complex64)
        Ht = Ht.pin_memory() if host else Ht.cuda()
        out.append((M, K, L, Yt, Ht))
    return out


@pytest.mark.parametrize("host", [False, True])
@pytest.mark.parametrize("dtype", ["fp16", "fp32", "e4m3"])
def test_grouped_equals_per_request(pk, dtype, host):
    r = 10
    bits = mseq.mseq_bits(r, 0)
    N = bits.size
    dev = torch.device("cuda", 0)
    pilot = pk.Pilot(bits, device=dev)
    specs = [(5, 2, 64), (64, 8, 32), (1, 1, 1), (130, 4, 100), (7, 15, 64)]
    reqs = _requests(N, specs, 1, host)
    rows = 256
    kl_max = 1000
    buf, arr = _table(pk, len(reqs) + 2)
    off = 0
    for i, (M, K, L, Y, H) in enumerate(reqs):
        arr[i].Y, arr[i].H, arr[i].M, arr[i].K, arr[i].L = Y.data_ptr(), H.data_ptr(), M, K, L
        arr[i].row_offset = off
        off += M
    # two empty slots at the end
    ws = torch.empty(pk.grouped_workspace_size(rows, N, kl_max, dtype), dtype=torch.uint8,
                     device=dev)
    pk.estimate_grouped(pilot, buf.data_ptr(), len(reqs) + 2, rows, kl_max, dtype, ws)
    torch.cuda.synchronize()
    assert pk.get_status(dev) == 0
    for M, K, L, Y, H in reqs:
        ref = pk.estimate(Y.cuda().view(1, M, N), pilot, K, L, dtype=dtype).reshape(M, K * L)
        if dtype == "fp32" and K * L <= 32:
            # alone, a request of few lags takes the few-lags FP32 kernel, whose sums run in
            # another order than the batch's tiled kernel: equal to FP32 rounding
            a, b = H.cpu().numpy(), ref.cpu().numpy()
            assert np.sum(np.abs(a - b) ** 2) <= 1e-12 * np.sum(np.abs(b) ** 2)
        else:
            assert torch.equal(H.cpu(), ref.cpu())


def test_grouped_invalid_descriptor_is_skipped(pk):
    bits = mseq.mseq_bits(9, 1)
    N = bits.size
    dev = torch.device("cuda", 0)
    pilot = pk.Pilot(bits, device=dev)
    reqs = _requests(N, [(8, 2, 16), (8, 2, 16)], 2, False)
    buf, arr = _table(pk, 2)
    for i, (M, K, L, Y, H) in enumerate(reqs):
        arr[i].Y, arr[i].H, arr[i].M, arr[i].K, arr[i].L = Y.data_ptr(), H.data_ptr(), M, K, L
    arr[0].row_offset = 0
    arr[1].row_offset = 60                     # 60 + 8 > 64 rows: invalid
    ws = torch.empty(pk.grouped_workspace_size(64, N, 32, "fp16"), dtype=torch.uint8, device=dev)
    pk.estimate_grouped(pilot, buf.data_ptr(), 2, 64, 32, "fp16", ws)
    torch.cuda.synchronize()
    assert pk.get_status(dev) == 1             # PNCE_EINVAL latched
    assert pk.get_status(dev) == 0             # and cleared by the read
    M, K, L, Y, H = reqs[0]
    ref = pk.estimate(Y.view(1, M, N), pilot, K, L, dtype="fp16").reshape(M, K * L)
    assert torch.equal(H, ref)
    assert torch.all(reqs[1][4] == complex(5.0, 5.0))      # untouched


def test_grouped_graph_replay_follows_descriptors(pk):
    bits = mseq.mseq_bits(8, 0)
    N = bits.size
    dev = torch.device("cuda", 0)
    pilot = pk.Pilot(bits, device=dev)
    rows, kl_max = 64, 64
    buf, arr = _table(pk, 4)
    ws = torch.empty(pk.grouped_workspace_size(rows, N, kl_max, "fp16"), dtype=torch.uint8,
                     device=dev)
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        pk.estimate_grouped(pilot, buf.data_ptr(), 4, rows, kl_max, "fp16", ws,
                            stream=s.cuda_stream)          # eager run sets kernel attributes
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pk.estimate_grouped(pilot, buf.data_ptr(), 4, rows, kl_max, "fp16", ws,
                            stream=torch.cuda.current_stream(dev).cuda_stream)
    for seed in (3, 4):
        reqs = _requests(N, [(3, 2, 16), (20, 4, 16), (9, 1, 64)], seed, True)
        off = 0
        for i, (M, K, L, Y, H) in enumerate(reqs):
            arr[i].Y, arr[i].H, arr[i].M, arr[i].K, arr[i].L = Y.data_ptr(), H.data_ptr(), M, K, L
            arr[i].row_offset = off
            off += M
        arr[3].M = 0
        with torch.cuda.stream(s):
            g.replay()
        s.synchronize()
        assert pk.get_status(dev) == 0
        for M, K, L, Y, H in reqs:
            ref = pk.estimate(Y.cuda().view(1, M, N), pilot, K, L, dtype="fp16").reshape(M, K * L)
            assert torch.equal(H, ref.cpu())


def test_grouped_overlapping_rows_latch_einval(pk):
    # two requests whose row ranges overlap (rows 4..7 claimed twice) are a caller error:
    # PNCE_EINVAL is latched; a third request elsewhere in the batch is unaffected
    bits = mseq.mseq_bits(9, 1)
    N = bits.size
    dev = torch.device("cuda", 0)
    pilot = pk.Pilot(bits, device=dev)
    reqs = _requests(N, [(8, 2, 16), (8, 2, 16), (6, 1, 32)], 7, True)
    buf, arr = _table(pk, 3)
    for i, (M, K, L, Y, H) in enumerate(reqs):
        arr[i].Y, arr[i].H, arr[i].M, arr[i].K, arr[i].L = Y.data_ptr(), H.data_ptr(), M, K, L
    arr[0].row_offset, arr[1].row_offset, arr[2].row_offset = 0, 4, 20
    for dtype in ("fp16", "fp32"):
        ws = torch.empty(pk.grouped_workspace_size(64, N, 32, dtype), dtype=torch.uint8,
                         device=dev)
        pk.estimate_grouped(pilot, buf.data_ptr(), 3, 64, 32, dtype, ws)
        torch.cuda.synchronize()
        assert pk.get_status(dev) == 1             # PNCE_EINVAL latched
        M, K, L, Y, H = reqs[2]
        ref = pk.estimate(Y.cuda().view(1, M, N), pilot, K, L, dtype=dtype).reshape(M, K * L)
        if dtype == "fp32":
            a, b = H.numpy(), ref.cpu().numpy()
            assert np.sum(np.abs(a - b) ** 2) <= 1e-12 * np.sum(np.abs(b) ** 2)
        else:
            assert torch.equal(H, ref.cpu())


@pytest.mark.parametrize("host", [False, True])
def test_grouped_auto_dtype(pk, host):
    # PNCE_AUTO resolves on kl_max: the FP32 path at <= 16 lags, fp16 tensor cores above
    bits = mseq.mseq_bits(10, 2)
    N = bits.size
    dev = torch.device("cuda", 0)
    pilot = pk.Pilot(bits, device=dev)
    for kl_max, want in ((16, "fp32"), (64, "fp16")):
        assert pk.lib().pnce_auto_dtype(N, 1, kl_max) == pk.DTYPES[want]
        assert pk.grouped_workspace_size(128, N, kl_max, "auto") == \
            pk.grouped_workspace_size(128, N, kl_max, want)
        outs = []
        for dtype in ("auto", want):
            reqs = _requests(N, [(40, 2, kl_max // 2), (17, 1, kl_max)], 3, host)
            buf, arr = _table(pk, 2)
            off = 0
            for i, (M, K, L, Y, H) in enumerate(reqs):
                arr[i].Y, arr[i].H, arr[i].M, arr[i].K, arr[i].L = \
                    Y.data_ptr(), H.data_ptr(), M, K, L
                arr[i].row_offset = off
                off += M
            ws = torch.empty(pk.grouped_workspace_size(128, N, kl_max, dtype), dtype=torch.uint8,
                             device=dev)
            pk.estimate_grouped(pilot, buf.data_ptr(), 2, 128, kl_max, dtype, ws)
            torch.cuda.synchronize()
            assert pk.get_status(dev) == 0
            outs.append([H.cpu() for *_, H in reqs])
        for a, b in zip(*outs):
            assert torch.equal(a, b)
