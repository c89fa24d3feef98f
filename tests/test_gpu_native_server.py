"""The native serving loop (pnce_server_*) on the GPU: a Poisson stream of uneven requests,
results checked against the oracle and bit-identical to the Python loop's (the same
grouped batches, the same kernels), a request whose PN length has no pilot failing alone,
and a tight memory cap."""
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
        reqs.append(serve.Request(s.rid, s.t_arrival, s.M, s.N, s.K, s.L,
                                  y.data_ptr() + s.slot * s.M * s.N * 8,
                                  out.data_ptr() + off * 8))
        reqs[-1].off = off
        off += s.M * s.K * s.L
    return reqs


def _result(out, r):
    return out[r.off:r.off + r.M * r.K * r.L].numpy().reshape(r.M, r.K, r.L)


@pytest.mark.parametrize("dtype", ["fp16", "fp32"])
def test_native_trace_matches_oracle_and_python_loop(setup, dtype):
    serve, pool, pinned = setup
    dev = torch.device("cuda", 0)
    specs = S.poisson_trace(20000.0, 0.03, seed=21, payload_slots=2)
    total = sum(s.M * s.K * s.L for s in specs)
    out_n = torch.zeros(total, dtype=torch.complex64, pin_memory=True)
    out_p = torch.zeros(total, dtype=torch.complex64, pin_memory=True)
    nat = serve.NativeServer(S.pilot_bits, device=dev, dtype=dtype, slots=3)
    nat.prepare(sorted({s.N for s in specs}), caps=(64, 256))
    reqs = _requests(serve, pinned, specs, out_n)
    st = nat.run(reqs)
    assert st["requests"] == len(reqs) and st["failed"] == 0
    assert st["batches"] < len(reqs)                 # requests were batched together
    for r in reqs:
        assert r.t_arrival <= r.t_admit <= r.t_launch < r.t_done and r.batch >= 0
    for r in reqs[::5]:
        Y = pool[(r.M, r.N)][[specs[r.rid].slot]]
        bits = S.pilot_bits(r.N)
        H = _result(out_n, r)[None]
        assert O.nmse(H, O.estimate(Y, bits, r.K, r.L)) <= TOL[dtype], r
        if dtype in TOL_Q:
            assert O.nmse(H, O.estimate_quantized(Y, bits, r.K, r.L, dtype)) <= TOL_Q[dtype]
    # the Python loop over the same trace: every result the same bits
    eng = serve.GpuEngine(S.pilot_bits, device=dev, dtype=dtype, slots=3)
    serve.Server(eng).run(_requests(serve, pinned, specs, out_p))
    assert torch.equal(out_n, out_p)


def test_native_missing_pilot_fails_only_its_requests(setup):
    serve, pool, pinned = setup
    dev = torch.device("cuda", 0)
    specs = S.poisson_trace(20000.0, 0.01, seed=22, payload_slots=2)
    Ns = sorted({s.N for s in specs})
    total = sum(s.M * s.K * s.L for s in specs)
    out = torch.zeros(total, dtype=torch.complex64, pin_memory=True)
    nat = serve.NativeServer(S.pilot_bits, device=dev, dtype="fp16", slots=2)
    for N in Ns[1:]:
        nat.pilot(N)
    reqs = _requests(serve, pinned, specs, out)
    # the run registers pilots for the trace's lengths itself; bypass that for one length
    from paper_2206_05506_gb300 import lib
    import ctypes as C
    table = serve._req_table(reqs)
    res = np.empty(len(reqs), dtype=serve.OUT_DTYPE)
    nb = C.c_int(0)
    st = lib().pnce_server_run(nat._s, table.ctypes.data, len(reqs), res.ctypes.data,
                               C.byref(nb))
    assert st == 0
    missing = np.array([r.N == Ns[0] for r in reqs])
    assert missing.any() and (~missing).any()
    assert np.all(res["status"][missing] == 1)       # PNCE_EINVAL: no pilot for that N
    assert np.all(res["status"][~missing] == 0)
    for r, o in zip(reqs, res):
        if o["status"] == 0:
            assert O.nmse(_result(out, r)[None],
                          O.estimate(pool[(r.M, r.N)][[specs[r.rid].slot]],
                                     S.pilot_bits(r.N), r.K, r.L)) <= TOL["fp16"]


def test_native_memory_cap(setup):
    serve, pool, pinned = setup
    dev = torch.device("cuda", 0)
    specs = S.poisson_trace(20000.0, 0.01, seed=23, payload_slots=2)
    total = sum(s.M * s.K * s.L for s in specs)
    out = torch.zeros(total, dtype=torch.complex64, pin_memory=True)
    nat = serve.NativeServer(S.pilot_bits, device=dev, dtype="fp16", slots=4,
                             mem_cap_bytes=8e6)
    reqs = _requests(serve, pinned, specs, out)
    st = nat.run(reqs)
    assert st["requests"] == len(reqs) and st["failed"] == 0
    assert any(r.t_admit > r.t_arrival for r in reqs)


def test_native_pilot_replacement_recaptures(setup):
    # a new pilot for an N drops the graphs captured with the old one, which may then go
    import gc
    from paper_2206_05506_gb300 import Pilot, lib
    serve, pool, pinned = setup
    dev = torch.device("cuda", 0)
    specs = [s for s in S.poisson_trace(20000.0, 0.01, seed=24, payload_slots=2)
             if s.N == 1023][:20]
    total = sum(s.M * s.K * s.L for s in specs)
    out = torch.zeros(total, dtype=torch.complex64, pin_memory=True)
    nat = serve.NativeServer(S.pilot_bits, device=dev, dtype="fp16", slots=2)
    nat.prepare([1023], caps=(64, 256))
    new = Pilot(S.pilot_bits(1023), device=dev)
    assert lib().pnce_server_add_pilot(nat._s, new.handle) == 0
    old, nat._pilots[1023] = nat._pilots[1023], new
    del old
    gc.collect()                                     # the old pilot's table is freed
    reqs = _requests(serve, pinned, specs, out)
    st = nat.run(reqs)
    assert st["requests"] == len(reqs) and st["failed"] == 0
    for r in reqs:
        ref = O.estimate(pool[(r.M, r.N)][[specs[reqs.index(r)].slot]], S.pilot_bits(r.N),
                         r.K, r.L)
        assert O.nmse(_result(out, r)[None], ref) <= TOL["fp16"]


def test_native_online_session(setup):
    # requests submitted one by one while earlier ones run, results collected by polling:
    # every ticket reported once, each result the oracle's, and a trace run refused while
    # the session has open requests
    from paper_2206_05506_gb300 import PnceError
    serve, pool, pinned = setup
    dev = torch.device("cuda", 0)
    specs = S.poisson_trace(20000.0, 0.004, seed=25, payload_slots=2)
    total = sum(s.M * s.K * s.L for s in specs)
    out = torch.zeros(total, dtype=torch.complex64, pin_memory=True)
    nat = serve.NativeServer(S.pilot_bits, device=dev, dtype="fp16", slots=3)
    nat.prepare(sorted({s.N for s in specs}), caps=(64, 256))
    reqs = _requests(serve, pinned, specs, out)
    nat.start()
    seen = {}
    tickets = []
    for k, r in enumerate(reqs):
        tickets.append(nat.submit(r))
        if k == 0:
            with pytest.raises(PnceError):            # the session shares the slots
                nat.run([r])
            with pytest.raises(PnceError):            # the session is still open
                nat.start()
        for t, o in nat.poll(max_out=4):
            seen[t] = o
    assert tickets == list(range(len(reqs)))
    for _ in range(100000):
        if nat.open_requests() == 0:
            break
        for t, o in nat.poll(max_out=4):
            assert t not in seen
            seen[t] = o
    assert nat.open_requests() == 0 and sorted(seen) == tickets
    for t, r in zip(tickets, reqs):
        o = seen[t]
        assert o["status"] == 0 and 0 <= o["t_admit"] <= o["t_launch"] < o["t_done"]
        ref = O.estimate(pool[(r.M, r.N)][[specs[t].slot]], S.pilot_bits(r.N), r.K, r.L)
        assert O.nmse(_result(out, r)[None], ref) <= TOL["fp16"]
    nat.start()                                       # a new session once all are reported
    assert nat.open_requests() == 0
