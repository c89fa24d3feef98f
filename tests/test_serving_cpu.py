"""Scheduling logic of the serving loop with a fake engine on a virtual clock (no GPU):
admission by memory, bucketing, batch packing, concurrency limit, latency accounting, and
batches whose engine calls raise (faults injected on the host)."""
import numpy as np

from paper_2206_05506_gb300.serve import CAPACITIES, Request, Server, kl_class
from synth import serving as S


class Clock:
    def __init__(self, dt=5e-6):
        self.t, self.dt = 0.0, dt

    def __call__(self):
        self.t += self.dt
        return self.t


class FakeEngine:
    """Each batch takes `base + per_row * rows` seconds of virtual time."""

    def __init__(self, clock, slots=2, base=200e-6, per_row=0.2e-6, nbytes=lambda r: r.M * 1000):
        self.clock, self.slots, self.base, self.per_row = clock, slots, base, per_row
        self.nbytes = nbytes
        self.launched = []
        self.running = 0
        self.max_running = 0

    def footprint(self, r):
        return self.nbytes(r)

    def launch(self, slot, N, klc, reqs):
        rows = sum(r.M for r in reqs)
        self.launched.append((slot, N, klc, [r.rid for r in reqs], rows))
        self.running += 1
        self.max_running = max(self.max_running, self.running)
        return {"end": self.clock.t + self.base + self.per_row * rows, "done": False}

    def done(self, tok):
        if not tok["done"] and self.clock.t >= tok["end"]:
            tok["done"] = True
            self.running -= 1
        return tok["done"]


def _requests(rate=20000.0, dur=0.02, seed=1):
    specs = S.poisson_trace(rate, dur, seed=seed)
    return [Request(s.rid, s.t_arrival, s.M, s.N, s.K, s.L, 0, 0) for s in specs]


def test_kl_classes():
    assert kl_class(16, 255) == 64 and kl_class(64, 255) == 64 and kl_class(65, 255) == 255
    assert kl_class(65, 1023) == 256 and kl_class(1000, 1023) == 1023
    assert kl_class(1024, 2047) == 1024 and kl_class(3, 2047) == 64


def test_all_requests_served_in_valid_batches():
    clock = Clock()
    eng = FakeEngine(clock, slots=3)
    srv = Server(eng, mem_cap_bytes=1e12, max_batch_rows=4096)
    reqs = _requests()
    st = srv.run(reqs, clock=clock, t0=0.0)
    assert st["requests"] == len(reqs) and len(srv.done) == len(reqs)
    byid = {r.rid: r for r in reqs}
    seen = set()
    for slot, N, klc, rids, rows in eng.launched:
        assert rows <= 4096 and rows == sum(byid[i].M for i in rids)
        for i in rids:
            r = byid[i]
            assert r.N == N and kl_class(r.K * r.L, r.N) == klc     # one bucket per batch
            assert klc >= r.K * r.L
            assert i not in seen
            seen.add(i)
    assert eng.max_running <= 3
    for r in reqs:
        assert r.t_arrival <= r.t_admit <= r.t_launch < r.t_done
    # FIFO inside a bucket
    order = {}
    for _, N, klc, rids, _ in eng.launched:
        order.setdefault((N, klc), []).extend(rids)
    for rids in order.values():
        assert rids == sorted(rids)


def test_batches_grow_under_load():
    # one slot and a slow engine: arrivals pile up and are served together
    clock = Clock()
    eng = FakeEngine(clock, slots=1, base=2e-3)
    srv = Server(eng, mem_cap_bytes=1e12)
    srv.run(_requests(dur=0.05), clock=clock, t0=0.0)
    assert np.mean([len(x[3]) for x in eng.launched]) > 1.5


def test_memory_cap_admission():
    clock = Clock()
    eng = FakeEngine(clock, slots=4, base=1e-3, nbytes=lambda r: r.M * 10_000)
    cap = 3_000_000                                    # room for ~ 1-4 requests at a time
    srv = Server(eng, mem_cap_bytes=cap)
    reqs = _requests(dur=0.01)
    srv.run(reqs, clock=clock, t0=0.0)
    assert len(srv.done) == len(reqs)
    assert srv.peak_inflight_bytes <= cap
    assert srv.inflight_bytes == 0
    assert any(r.t_admit > r.t_arrival + 1e-4 for r in reqs)   # some had to wait


def test_latency_stats():
    clock = Clock()
    eng = FakeEngine(clock, slots=2)
    srv = Server(eng)
    st = srv.run(_requests(dur=0.01), clock=clock, t0=0.0)
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    assert st["p50_ms"] >= 0.2                        # at least one batch service time
    assert st["frames_per_s"] > 0 and st["taps_per_s"] > 0


def test_poisson_trace_shapes():
    specs = S.poisson_trace(20000.0, 0.5, seed=3)
    assert abs(len(specs) / 0.5 - 20000.0) < 5 * np.sqrt(20000.0 * 0.5) / 0.5
    for s in specs:
        assert s.M in S.M_CHOICES and s.N in (255, 511, 1023, 2047) and s.L in S.L_CHOICES
        assert 1 <= s.K <= min(s.N // s.L, 16) and s.K * s.L <= s.N
    t = np.array([s.t_arrival for s in specs])
    assert np.all(np.diff(t) > 0)
    assert CAPACITIES[-1] >= 4096


class FlakyEngine(FakeEngine):
    """Every `launch_every`-th launch raises; every `done_every`-th launched batch raises
    when it completes (a device error reported at completion)."""

    def __init__(self, clock, launch_every=5, done_every=7, **kw):
        super().__init__(clock, **kw)
        self.launch_every, self.done_every = launch_every, done_every
        self.calls = 0
        self.ok = 0

    def launch(self, slot, N, klc, reqs):
        self.calls += 1
        if self.calls % self.launch_every == 0:
            raise RuntimeError("launch refused")
        tok = super().launch(slot, N, klc, reqs)
        self.ok += 1
        tok["fault"] = self.ok % self.done_every == 0
        return tok

    def done(self, tok):
        fin = super().done(tok)
        if fin and tok["fault"]:
            raise RuntimeError("device error at completion")
        return fin


def test_failing_batches_are_reported_and_the_loop_goes_on():
    clock = Clock()
    eng = FlakyEngine(clock, slots=3)
    srv = Server(eng, mem_cap_bytes=2e6, max_batch_rows=1024)
    reqs = _requests(dur=0.03, seed=5)
    st = srv.run(reqs, clock=clock, t0=0.0)
    ok = {r.rid for r in srv.done}
    bad = {r.rid for r in srv.failed}
    assert ok.isdisjoint(bad) and ok | bad == {r.rid for r in reqs}
    assert st["failed"] == len(bad) > 0 and st["requests"] == len(ok) > 0
    assert all(r.error.startswith("RuntimeError") for r in srv.failed)
    assert all(r.error == "" and r.t_done >= r.t_arrival for r in srv.done)
    # every byte and every stream slot came back
    assert srv.inflight_bytes == 0
    assert sorted(srv.free_slots) == list(range(eng.slots)) and not srv.busy


class LatchingEngine(FakeEngine):
    """Reports, when asked at the end of a run, an error latched on the device."""

    def check(self):
        raise RuntimeError("device status: a wait ran out")


def test_a_latched_device_error_is_raised_at_the_end_of_the_run():
    import pytest
    clock = Clock()
    eng = LatchingEngine(clock, slots=2)
    srv = Server(eng)
    reqs = _requests(dur=0.005)
    with pytest.raises(RuntimeError, match="wait ran out"):
        srv.run(reqs, clock=clock, t0=0.0)
    assert len(srv.done) == len(reqs)          # every batch ran before the check
