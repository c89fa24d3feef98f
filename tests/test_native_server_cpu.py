"""The native serving loop's scheduling (pnce_sched_simulate: the C++ scheduler on a virtual
clock, no GPU) makes exactly the decisions of the Python Server with the fake engine of
test_serving_cpu on the same clock: same admission, launch and completion times, same
batches."""
import numpy as np
import pytest

from paper_2206_05506_gb300 import PnceError
from paper_2206_05506_gb300.serve import Request, Server, simulate
from synth import serving as S
from test_serving_cpu import Clock, FakeEngine


def _trace(rate, dur, seed):
    specs = S.poisson_trace(rate, dur, seed=seed)
    return [Request(s.rid, s.t_arrival, s.M, s.N, s.K, s.L, 0, 0) for s in specs]


@pytest.mark.parametrize("slots,cap,rows,base,seed", [
    (3, 1e12, 4096, 200e-6, 1),          # plenty of memory
    (1, 1e12, 4096, 2e-3, 2),            # one slow slot: batches grow
    (4, 3_000_000, 4096, 1e-3, 3),       # tight memory: admission waits
    (2, 1e12, 300, 400e-6, 4),           # small batches: packing limit
])
def test_simulation_matches_python_scheduler(slots, cap, rows, base, seed):
    py = _trace(20000.0, 0.02, seed)
    clock = Clock()
    eng = FakeEngine(clock, slots=slots, base=base)
    srv = Server(eng, mem_cap_bytes=cap, max_batch_rows=rows)
    srv.run(py, clock=clock, t0=0.0)
    out, nb = simulate(_trace(20000.0, 0.02, seed), slots, cap, rows, row_bytes=1000.0,
                       base_s=base, per_row_s=0.2e-6, clock_dt=5e-6)
    assert nb == srv.batches == len(eng.launched)
    assert np.all(out["status"] == 0)
    np.testing.assert_array_equal(out["t_admit"], [r.t_admit for r in py])
    np.testing.assert_array_equal(out["t_launch"], [r.t_launch for r in py])
    np.testing.assert_array_equal(out["t_done"], [r.t_done for r in py])
    np.testing.assert_array_equal(out["batch"], [r.batch for r in py])
    # each native batch holds the same requests as the Python one, in order
    for b, (_, N, klc, rids, _) in enumerate(eng.launched):
        assert list(np.flatnonzero(out["batch"] == b)) == rids


def test_simulation_rejects_invalid_traces():
    reqs = _trace(20000.0, 0.005, 5)
    with pytest.raises(PnceError):
        simulate(reqs, 0, 1e12)                       # no slot
    bad = list(reqs)
    bad[0], bad[1] = bad[1], bad[0]                   # arrivals out of order
    with pytest.raises(PnceError):
        simulate(bad, 2, 1e12)
    r = reqs[0]
    over = [Request(0, 0.0, r.M, r.N, r.N, 2, 0, 0)]  # K*L > N
    with pytest.raises(PnceError):
        simulate(over, 2, 1e12)
    out, nb = simulate([], 2, 1e12)
    assert nb == 0 and out.size == 0


def test_simulated_faults_match_python_loop():
    # batches whose launch is refused or that fail at completion (faults made on the host):
    # the same requests fail, at the same times, and every slot and byte comes back
    from test_serving_cpu import FlakyEngine
    py = _trace(20000.0, 0.03, 5)
    clock = Clock()
    eng = FlakyEngine(clock, slots=3)
    srv = Server(eng, mem_cap_bytes=2e6, max_batch_rows=1024)
    srv.run(py, clock=clock, t0=0.0)
    out, nb = simulate(_trace(20000.0, 0.03, 5), 3, 2e6, 1024, fail_launch_every=5,
                       fail_done_every=7)
    failed = {r.rid for r in srv.failed}
    assert failed and len(failed) < len(py)
    assert set(np.flatnonzero(out["status"] != 0)) == failed
    assert np.all(out["status"][list(failed)] == 4)          # PNCE_ECUDA
    np.testing.assert_array_equal(out["t_done"], [r.t_done for r in py])
    np.testing.assert_array_equal(out["t_launch"], [r.t_launch for r in py])
    assert nb == srv.batches


def test_native_stats_by_hand():
    # three requests: two in batch 0, one in batch 1, one of them failed; latencies 1 ms
    # and 3 ms for the two that finished
    from paper_2206_05506_gb300 import serve
    reqs = [Request(0, 0.000, 64, 255, 1, 16, 0, 0), Request(1, 0.001, 32, 255, 2, 16, 0, 0),
            Request(2, 0.002, 128, 511, 1, 64, 0, 0)]
    out = np.zeros(3, dtype=serve.OUT_DTYPE)
    out["t_admit"] = [0.0, 0.001, 0.002]
    out["t_launch"] = [0.0005, 0.0015, 0.0025]
    out["t_done"] = [0.001, 0.004, 0.003]
    out["batch"] = [0, 0, 1]
    out["status"] = [0, 0, 4]
    st = serve._native_stats(reqs, out, 2)
    assert st["requests"] == 2 and st["failed"] == 1 and st["batches"] == 2
    assert abs(st["mean_batch_rows"] - (96 + 128) / 2) < 1e-12
    assert abs(st["max_ms"] - 3.0) < 1e-9 and abs(st["p50_ms"] - 2.0) < 1e-9
    assert abs(st["frames_per_s"] - 2 / 0.004) < 1e-6
    assert abs(st["taps_per_s"] - (64 * 16 + 32 * 32) / 0.004) < 1e-3
    assert reqs[2].error == "status 4" and reqs[0].error == "" and reqs[1].batch == 0
    assert reqs[1].t_done == 0.004
