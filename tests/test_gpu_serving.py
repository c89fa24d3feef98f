"""Serving form on the GPU: a Poisson stream of uneven requests through the continuous
batching loop (CUDA-graph replays, several batches in flight), results checked against
the oracle, and each result identical alone and in the mix."""
import numpy as np
import pytest
import torch

from oracle import pn_oracle as O
from synth import serving as S

pytestmark = pytest.mark.gpu

TOL = {"fp16": 2e-3, "fp32": 1e-6}
TOL_Q = {"fp16": 1e-9}


@pytest.fixture(scope="module")
def setup():
    from paper_2206_05506_gb300 import serve
    pool = S.payload_pool(slots=2, seed=4)
    pinned = {k: torch.from_numpy(v).pin_memory() for k, v in pool.items()}
    return serve, pool, pinned


def _requests(serve, pinned, specs, out):
    reqs, off = [], 0
    for s in specs:
        y = pinned[(s.M, s.N)]
        n = s.M * s.K * s.L
        reqs.append(serve.Request(s.rid, s.t_arrival, s.M, s.N, s.K, s.L,
                                  y.data_ptr() + s.slot * s.M * s.N * 8,
                                  out.data_ptr() + off * 8))
        reqs[-1].off = off
        off += n
    return reqs


def _result(out, r):
    return out[r.off:r.off + r.M * r.K * r.L].numpy().reshape(r.M, r.K, r.L)


@pytest.mark.parametrize("dtype", ["fp16", "fp32"])
def test_trace_results_and_mix_identity(setup, dtype):
    serve, pool, pinned = setup
    dev = torch.device("cuda", 0)
    eng = serve.GpuEngine(S.pilot_bits, device=dev, dtype=dtype, slots=3)
    specs = S.poisson_trace(20000.0, 0.03, seed=11, payload_slots=2)
    total = sum(s.M * s.K * s.L for s in specs)
    out = torch.zeros(total, dtype=torch.complex64, pin_memory=True)
    reqs = _requests(serve, pinned, specs, out)
    srv = serve.Server(eng, mem_cap_bytes=40e9)
    st = srv.run(reqs)
    assert st["requests"] == len(reqs)
    assert st["batches"] < len(reqs)                 # requests were batched together
    assert pytest.approx(0) == srv.inflight_bytes
    for r in reqs[::7]:
        Y = pool[(r.M, r.N)][[specs[r.rid].slot]]
        bits = S.pilot_bits(r.N)
        H = _result(out, r)[None]
        ref = O.estimate(Y, bits, r.K, r.L)
        assert O.nmse(H, ref) <= TOL[dtype], r
        if dtype in TOL_Q:
            assert O.nmse(H, O.estimate_quantized(Y, bits, r.K, r.L, dtype)) <= TOL_Q[dtype]
    # the same requests served alone (batch of one, rows at offset 0) give the same bits
    mixed = [r for r in reqs if r.batch >= 0][:: max(1, len(reqs) // 12)]
    for r in mixed:
        out2 = torch.zeros(r.M * r.K * r.L, dtype=torch.complex64, pin_memory=True)
        alone = serve.Request(r.rid, 0.0, r.M, r.N, r.K, r.L, r.y_addr, out2.data_ptr())
        serve.Server(eng).run([alone])
        a = out2.numpy().reshape(r.M, r.K, r.L)
        m = _result(out, r)
        assert O.nmse(a[None], m[None]) <= TOL_Q.get(dtype, 1e-9)
        assert np.array_equal(a, m), "result depends on its batch"


def test_memory_admission_cap(setup):
    serve, pool, pinned = setup
    dev = torch.device("cuda", 0)
    eng = serve.GpuEngine(S.pilot_bits, device=dev, dtype="fp16", slots=4)
    specs = S.poisson_trace(20000.0, 0.01, seed=12, payload_slots=2)
    out = torch.zeros(sum(s.M * s.K * s.L for s in specs), dtype=torch.complex64, pin_memory=True)
    reqs = _requests(serve, pinned, specs, out)
    cap = 12e6
    srv = serve.Server(eng, mem_cap_bytes=cap)
    st = srv.run(reqs)
    assert st["requests"] == len(reqs)
    assert srv.peak_inflight_bytes <= cap
    assert srv.inflight_bytes == 0
