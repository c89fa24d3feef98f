"""End-to-end estimate from host buffers (pnce_estimate_host) against the device path and
the oracle: page-locked buffers (copy-out by kernel) and pageable ones (copy-out by DMA),
batches that split into several double-buffered chunks with a ragged last chunk, every
arithmetic."""
import numpy as np
import pytest
import torch

from oracle import pn_oracle as O
from synth import channel as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    import paper_2206_05506_gb300 as pk
    pk.lib()
    return pk


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("dtype", ["fp32", "fp16", "e4m3", "tf32"])
@pytest.mark.parametrize("shape", [(7, 8, 2, 16, 3), (10, 37, 4, 100, 13), (12, 130, 8, 256, 9)])
def test_host_path_equals_device_path(pk, shape, dtype, pinned):
    r, M, K, L, F = shape
    w = C.Workload("t", r=r, M=M, K=K, L=L, F=F, snr_db=(10.0,), seed=r)
    bits, _, Y = C.make(w)
    dev = torch.device("cuda", 0)
    pilot = pk.Pilot(bits, device=dev)
    Yh = torch.from_numpy(Y)
    Yh = Yh.pin_memory() if pinned else Yh.clone()
    Hh = torch.full((F, M, K, L), complex(3.0, 3.0), dtype=torch.complex64)
    Hh = Hh.pin_memory() if pinned else Hh
    pk.estimate_host(Yh, pilot, K, L, dtype=dtype, out=Hh)
    assert pk.get_status(dev) == 0
    Hd = pk.estimate(Yh.to(dev), pilot, K, L, dtype=dtype).cpu()
    assert torch.equal(Hh, Hd)
    tol = {"fp32": 1e-6, "tf32": 1e-6, "fp16": 2e-3, "e4m3": 3e-2}[dtype]
    assert O.nmse(Hh.numpy(), O.estimate(Y, bits, K, L)) <= tol


def test_host_path_many_chunks(pk):
    # frames of 4 MB: the pipeline cuts 130 frames into chunks of ~31 with a ragged tail
    w = C.Workload("t", r=12, M=128, K=4, L=64, F=130, snr_db=(10.0,), seed=4)
    bits, _, Y = C.make(w)
    dev = torch.device("cuda", 0)
    pilot = pk.Pilot(bits, device=dev)
    Yh = torch.from_numpy(Y).pin_memory()
    Hh = torch.empty((130, 128, 4, 64), dtype=torch.complex64).pin_memory()
    pk.estimate_host(Yh, pilot, 4, 64, dtype="fp16", out=Hh)
    Hd = pk.estimate(Yh.to(dev), pilot, 4, 64, dtype="fp16").cpu()
    assert torch.equal(Hh, Hd)


def test_failure_part_way_leaves_no_work_in_flight(pk, monkeypatch):
    # a call that gives up at chunk 3 (a failure injected on the host, as a failed launch
    # or copy there would) still makes the caller's stream wait for the three chunks it had
    # enqueued: once that stream is synchronised, their results are complete in H and no
    # copy is still writing to it
    w = C.Workload("t", r=12, M=128, K=4, L=64, F=130, snr_db=(10.0,), seed=4)
    bits, _, Y = C.make(w)
    dev = torch.device("cuda", 0)
    pilot = pk.Pilot(bits, device=dev)
    Yh = torch.from_numpy(Y).pin_memory()
    sentinel = complex(3.0, -3.0)
    Hh = torch.full((130, 128, 4, 64), sentinel, dtype=torch.complex64).pin_memory()
    monkeypatch.setenv("PNCE_TEST_HOST_FAIL_CHUNK", "3")
    with pytest.raises(pk.PnceError):
        pk.estimate_host(Yh, pilot, 4, 64, dtype="fp16", out=Hh)
    torch.cuda.current_stream(dev).synchronize()
    monkeypatch.delenv("PNCE_TEST_HOST_FAIL_CHUNK")
    Hd = pk.estimate(Yh.to(dev), pilot, 4, 64, dtype="fp16").cpu()
    done = [bool(torch.equal(Hh[f], Hd[f])) for f in range(130)]
    untouched = [bool((Hh[f] == sentinel).all()) for f in range(130)]
    n = sum(done)
    assert n > 0 and n % 3 == 0 and all(done[:n])          # three whole chunks, in order
    assert all(untouched[n:])                               # nothing after them
    assert pk.get_status(dev) == 0
