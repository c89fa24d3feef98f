"""Continuous-batching estimation server.

Requests are single frames of uneven shape (M antennas, PN length N, K transmitters, L
taps) whose received blocks sit in page-locked host memory.  The loop

* admits arrivals while the bytes of admitted, unfinished work stay under a memory cap;
* buckets admitted requests by (N, lag class) -- requests of one bucket share a pilot and
  a padded lag count, so their antennas can be estimated as one batch;
* whenever a stream slot is free, launches the bucket whose oldest request has waited
  longest, packing as many of its requests as fit one batch: requests that arrive while
  other batches are on the GPU join the next batch, and up to `slots` batches run
  concurrently on their own streams;
* runs each batch as one replay of a CUDA graph captured once per (slot, N, lag class,
  capacity) around one pnce_estimate_grouped call: from a descriptor table in page-locked
  host memory it gathers the requests' antenna rows from host memory into the batch
  buffer, estimates (quantise + tensor-core correlation, or the FP32 SIMT path) and
  scatters each antenna's lags straight into its request's host result buffer;
* polls the batches' events and stamps each request's completion; latency is completion
  minus scheduled arrival;
* if the engine raises while launching or polling a batch, that batch's requests are
  recorded as failed (with the error), their memory and stream slot are released, and the
  loop goes on with the rest;
* at the end of a run it asks the engine (if the engine can tell) whether any kernel
  latched an error on the device -- a bounded wait that ran out, an invalid descriptor --
  and raises if one did, since some results may then be wrong.

Pilot tables and the per-shape buffers stay resident on the device.  Each request's result
depends only on its own antenna rows (per-antenna scales, fixed reduction order), so it is
the same alone and in any mix.

NativeServer runs the same rules inside the library (pnce_server_run, C++): a Python loop
spends tens of microseconds of host time per batch (descriptor table, graph replay, event),
which bounds the batches per second it can start; the native loop spends a few.  Server
stays for engines written in Python (and the fault-injection tests).
"""
from __future__ import annotations

import collections
import ctypes as C
import gc
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import (DTYPES, Pilot, _lib, check, context, estimate_grouped, grouped_workspace_size,
               lib)

KL_CLASSES = (64, 256, 1024)
CAPACITIES = (64, 256, 1024, 4096)        # antennas per batch


def kl_class(KL: int, N: int) -> int:
    for c in KL_CLASSES:
        if c >= KL:
            return min(c, N)
    return min(((KL + 1023) // 1024) * 1024, N)


@dataclass
class Request:
    rid: int
    t_arrival: float
    M: int
    N: int
    K: int
    L: int
    y_addr: int               # address of complex64 [M][N] (host page-locked or device)
    h_addr: int               # address of complex64 [M][K*L] for the result
    nbytes: int = 0
    t_admit: float = -1.0
    t_launch: float = -1.0
    t_done: float = -1.0
    batch: int = -1
    error: str = ""


@dataclass
class _Busy:
    slot: int
    token: object
    reqs: list
    bid: int


class Server:
    """Scheduling and admission, independent of how a batch is executed (`engine`)."""

    def __init__(self, engine, mem_cap_bytes: float = 40e9, max_batch_rows: int = 4096):
        self.engine = engine
        self.cap = float(mem_cap_bytes)
        self.max_rows = max_batch_rows
        self.pending: collections.deque = collections.deque()
        self.buckets: dict[tuple, collections.deque] = {}
        self.inflight_bytes = 0
        self.peak_inflight_bytes = 0
        self.free_slots = list(range(engine.slots))[::-1]
        self.busy: list[_Busy] = []
        self.done: list[Request] = []
        self.failed: list[Request] = []
        self.batches = 0
        self.batch_rows: list[int] = []

    # -- arrivals and admission
    def submit(self, req: Request):
        req.nbytes = self.engine.footprint(req)
        self.pending.append(req)

    def _admit(self, now: float):
        while self.pending:
            r = self.pending[0]
            if self.inflight_bytes + r.nbytes > self.cap and self.inflight_bytes > 0:
                break                                   # wait for memory to free up
            self.pending.popleft()
            self.inflight_bytes += r.nbytes
            self.peak_inflight_bytes = max(self.peak_inflight_bytes, self.inflight_bytes)
            r.t_admit = now
            key = (r.N, kl_class(r.K * r.L, r.N))
            self.buckets.setdefault(key, collections.deque()).append(r)

    def _fail(self, reqs: list, slot: int, now: float, exc: Exception):
        for r in reqs:
            r.t_done = now
            r.error = f"{type(exc).__name__}: {exc}"
            self.inflight_bytes -= r.nbytes
            self.failed.append(r)
        self.free_slots.append(slot)

    # -- completions
    def _complete(self, now: float):
        still = []
        for b in self.busy:
            try:
                finished = self.engine.done(b.token)
            except Exception as exc:                   # noqa: BLE001 -- reported per request
                self._fail(b.reqs, b.slot, now, exc)
                continue
            if finished:
                for r in b.reqs:
                    r.t_done = now
                    self.inflight_bytes -= r.nbytes
                    self.done.append(r)
                self.free_slots.append(b.slot)
            else:
                still.append(b)
        self.busy = still

    # -- launches
    def _launch(self, now: float):
        while self.free_slots:
            heads = [(q[0].t_arrival, key) for key, q in self.buckets.items() if q]
            if not heads:
                return
            _, key = min(heads)
            q = self.buckets[key]
            reqs, rows = [], 0
            while q and rows + q[0].M <= self.max_rows:
                r = q.popleft()
                reqs.append(r)
                rows += r.M
            if not reqs:                               # a single request above max_rows
                reqs.append(q.popleft())
                rows = reqs[0].M
            slot = self.free_slots.pop()
            for r in reqs:
                r.t_launch = now
                r.batch = self.batches
            try:
                token = self.engine.launch(slot, key[0], key[1], reqs)
            except Exception as exc:                   # noqa: BLE001 -- reported per request
                self._fail(reqs, slot, now, exc)
                continue
            self.busy.append(_Busy(slot, token, reqs, self.batches))
            self.batches += 1
            self.batch_rows.append(rows)

    def poll(self, now: float):
        self._complete(now)
        self._admit(now)
        self._launch(now)

    def idle(self) -> bool:
        return not (self.pending or self.busy or any(self.buckets.values()))

    def run(self, requests: list, clock=time.perf_counter, t0: float | None = None):
        """Open loop: each request is submitted at its t_arrival (seconds from t0).

        Python's cyclic garbage collector is paused while the loop runs: its collections
        of the many request objects stall the loop for milliseconds at a time, which shows
        up directly in the latency tail.  (Reference counting still frees everything the
        loop drops.)
        """
        t0 = clock() if t0 is None else t0
        i, n = 0, len(requests)
        gc_was_on = gc.isenabled()
        gc.disable()
        try:
            while i < n or not self.idle():
                now = clock() - t0
                while i < n and requests[i].t_arrival <= now:
                    self.submit(requests[i])
                    i += 1
                self.poll(now)
        finally:
            if gc_was_on:
                gc.enable()
        engine_check = getattr(self.engine, "check", None)
        if engine_check is not None:
            engine_check()
        return self.stats()

    def stats(self) -> dict:
        lat = np.array([r.t_done - r.t_arrival for r in self.done])
        if lat.size == 0:
            return {"requests": 0, "failed": len(self.failed)}
        t_first = min(r.t_arrival for r in self.done)
        t_last = max(r.t_done for r in self.done)
        taps = sum(r.M * r.K * r.L for r in self.done)
        span = max(t_last - t_first, 1e-9)
        return {"requests": int(lat.size), "batches": self.batches,
                "mean_batch_rows": float(np.mean(self.batch_rows)) if self.batch_rows else 0.0,
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "max_ms": float(lat.max() * 1e3),
                "frames_per_s": lat.size / span, "taps_per_s": taps / span,
                "peak_inflight_bytes": int(self.peak_inflight_bytes),
                "failed": len(self.failed)}


class _Shape:
    """Device buffers, descriptor tables and the captured graph of one batch shape."""

    def __init__(self, eng: "GpuEngine", slot: int, N: int, klc: int, cap: int):
        dev = eng.device
        self.N, self.klc, self.cap = N, klc, cap
        self.ws = torch.empty(grouped_workspace_size(cap, N, klc, eng.dtype), dtype=torch.uint8,
                              device=dev)
        # request descriptors (pnce_req_desc) in page-locked host memory: the kernels read
        # them directly, so a captured graph picks up each batch's table
        assert C.sizeof(_lib.ReqDesc) == 32
        self.desc = torch.zeros(cap * 32, dtype=torch.uint8, pin_memory=True)
        d = self.desc.numpy()
        self.d_ptr = d.view(np.int64).reshape(cap, 4)      # Y, H
        self.d_int = d.view(np.int32).reshape(cap, 8)      # [4] M, [5] K, [6] L, [7] row offset
        self.pilot = eng.pilot(N)
        self.graph = None
        stream = eng.streams[slot]
        if eng.use_graphs:
            with torch.cuda.stream(stream):
                self._enqueue(eng, stream.cuda_stream)      # eager run: sets kernel attributes
            stream.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                self._enqueue(eng, torch.cuda.current_stream(dev).cuda_stream)
            self.graph = g

    def _enqueue(self, eng: "GpuEngine", s: int):
        estimate_grouped(self.pilot, self.desc.data_ptr(), self.cap, self.cap, self.klc, eng.dtype,
                         self.ws, stream=s)

    def run(self, eng: "GpuEngine", slot: int, reqs: list):
        n = len(reqs)
        self.d_ptr[:n, 0] = [r.y_addr for r in reqs]
        self.d_ptr[:n, 1] = [r.h_addr for r in reqs]
        self.d_int[:n, 4] = [r.M for r in reqs]
        self.d_int[:n, 5] = [r.K for r in reqs]
        self.d_int[:n, 6] = [r.L for r in reqs]
        self.d_int[:n, 7] = np.cumsum([0] + [r.M for r in reqs[:-1]])
        self.d_int[n:, 4] = 0                              # empty slots
        stream = eng.streams[slot]
        with torch.cuda.stream(stream):
            if self.graph is not None:
                self.graph.replay()
            else:
                self._enqueue(eng, stream.cuda_stream)


class GpuEngine:
    """Executes batches with libpnce on one device: `slots` streams, graphs per shape."""

    def __init__(self, pilot_bits, device=None, dtype="fp16", slots: int = 3,
                 use_graphs: bool = True):
        """pilot_bits: callable N -> 0/1 array, the m-sequence used for PN length N."""
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index)
        self.dt = DTYPES[dtype]
        self.dtype = dtype
        self.slots = slots
        self.use_graphs = use_graphs
        self.ctx = context(self.device)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(slots)]
        self.events = [torch.cuda.Event() for _ in range(slots)]
        self._pilots: dict[int, Pilot] = {}
        self._shapes: dict[tuple, _Shape] = {}
        self._pilot_bits = pilot_bits
        self.elt = {0: 0, 1: 4, 2: 2, 3: 2, 4: 1}[self.dt]

    def pilot(self, N: int) -> Pilot:
        if N not in self._pilots:
            self._pilots[N] = Pilot(self._pilot_bits(N), device=self.device)
        return self._pilots[N]

    def footprint(self, r: Request) -> int:
        pitch = (r.N + 63) // 64 * 64
        return r.M * (8 * r.N + 2 * self.elt * pitch + 8 * kl_class(r.K * r.L, r.N))

    def prepare(self, Ns, caps=CAPACITIES[:3]):
        """Create (and capture) the batch shapes of every (N, lag class) bucket of the given
        PN lengths, for every slot, before serving starts."""
        for N in Ns:
            for klc in sorted({kl_class(k, N) for k in KL_CLASSES if k <= N} | {kl_class(N, N)}):
                for slot in range(self.slots):
                    for c in caps:
                        self._shape(slot, N, klc, c)

    def _shape(self, slot, N, klc, cap) -> _Shape:
        key = (slot, N, klc, cap)
        if key not in self._shapes:
            with torch.cuda.device(self.device):
                self._shapes[key] = _Shape(self, slot, N, klc, cap)
        return self._shapes[key]

    def launch(self, slot: int, N: int, klc: int, reqs: list):
        rows = sum(r.M for r in reqs)
        cap = next((c for c in CAPACITIES if c >= rows), None)
        if cap is None:
            cap = (rows + 4095) // 4096 * 4096
        shape = self._shape(slot, N, klc, cap)
        shape.run(self, slot, reqs)
        ev = self.events[slot]
        ev.record(self.streams[slot])
        return ev

    @staticmethod
    def done(token) -> bool:
        return token.query()

    def check(self):
        """Raise PnceError if a kernel of the batches run so far latched an error status
        (reads and clears the handle's status word; waits for the device)."""
        torch.cuda.synchronize(self.device)
        check(self.ctx.status(), "serving batches")


# Request and result tables of the native loop (pnce_serve_req / pnce_serve_out)
REQ_DTYPE = np.dtype([("Y", np.uint64), ("H", np.uint64), ("M", np.int32), ("N", np.int32),
                      ("K", np.int32), ("L", np.int32), ("t_arrival", np.float64)])
OUT_DTYPE = np.dtype([("t_admit", np.float64), ("t_launch", np.float64),
                      ("t_done", np.float64), ("batch", np.int32), ("status", np.int32)])
assert REQ_DTYPE.itemsize == C.sizeof(_lib.ServeReq) and OUT_DTYPE.itemsize == C.sizeof(_lib.ServeOut)


def _req_table(requests: list) -> np.ndarray:
    a = np.empty(len(requests), dtype=REQ_DTYPE)
    a["Y"] = [r.y_addr for r in requests]
    a["H"] = [r.h_addr for r in requests]
    a["M"] = [r.M for r in requests]
    a["N"] = [r.N for r in requests]
    a["K"] = [r.K for r in requests]
    a["L"] = [r.L for r in requests]
    a["t_arrival"] = [r.t_arrival for r in requests]
    return a


def _native_stats(requests: list, out: np.ndarray, batches: int) -> dict:
    """Write the run's times into the Request objects and summarise them as Server.stats
    does."""
    ok = out["status"] == 0
    for r, o in zip(requests, out):
        r.t_admit, r.t_launch, r.t_done = float(o["t_admit"]), float(o["t_launch"]), float(o["t_done"])
        r.batch = int(o["batch"])
        r.error = "" if o["status"] == 0 else f"status {int(o['status'])}"
    if not ok.any():
        return {"requests": 0, "failed": int((~ok).sum())}
    t_arr = np.array([r.t_arrival for r in requests])
    M = np.array([r.M for r in requests], dtype=np.float64)
    KL = np.array([r.K * r.L for r in requests], dtype=np.float64)
    lat = (out["t_done"] - t_arr)[ok]
    span = max(float(out["t_done"][ok].max() - t_arr[ok].min()), 1e-9)
    launched = out["batch"] >= 0
    rows = np.bincount(out["batch"][launched], weights=M[launched], minlength=batches)[:batches]
    return {"requests": int(lat.size), "batches": int(batches),
            "mean_batch_rows": float(rows.mean()) if batches else 0.0,
            "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "max_ms": float(lat.max() * 1e3),
            "frames_per_s": lat.size / span, "taps_per_s": float((M * KL)[ok].sum()) / span,
            "failed": int((~ok).sum())}


def simulate(requests: list, slots: int, mem_cap_bytes: float, max_batch_rows: int = 4096,
             row_bytes: float = 1000.0, base_s: float = 200e-6, per_row_s: float = 0.2e-6,
             clock_dt: float = 5e-6, fail_launch_every: int = 0, fail_done_every: int = 0):
    """The native loop's scheduling on a virtual clock, no GPU (pnce_sched_simulate):
    returns (per-request results as OUT_DTYPE, number of batches).  fail_*_every: faults
    made on the host (every n-th launch refused, every n-th started batch failing when it
    completes)."""
    reqs = _req_table(requests)
    out = np.empty(len(requests), dtype=OUT_DTYPE)
    nb = C.c_int(0)
    check(lib().pnce_sched_simulate(reqs.ctypes.data, len(requests), slots,
                                         float(mem_cap_bytes), max_batch_rows, float(row_bytes),
                                         float(base_s), float(per_row_s), float(clock_dt),
                                         int(fail_launch_every), int(fail_done_every),
                                         out.ctypes.data, C.byref(nb)), "pnce_sched_simulate")
    return out, nb.value


class NativeServer:
    """The serving loop run inside the library (pnce_server_*): the scheduling rules of
    Server, with the host side of each batch -- its descriptor table, the graph launch and
    the completion event -- in C++.  Requests as for Server; run() replays them open loop
    on the calling thread and returns the same statistics."""

    def __init__(self, pilot_bits, device=None, dtype: str = "fp16", slots: int = 8,
                 mem_cap_bytes: float = 40e9, max_batch_rows: int = 4096):
        self.ctx = context(device)
        self.device = self.ctx.device
        self.dtype, self.slots = dtype, slots
        self._pilot_bits = pilot_bits
        self._pilots: dict[int, Pilot] = {}
        p = C.c_void_p()
        with torch.cuda.device(self.device):
            check(lib().pnce_server_create(self.ctx.handle, DTYPES[dtype], slots,
                                                float(mem_cap_bytes), max_batch_rows,
                                                C.byref(p)), "pnce_server_create")
        self._s = p

    def pilot(self, N: int) -> Pilot:
        if N not in self._pilots:
            pl = Pilot(self._pilot_bits(N), device=self.device)
            check(lib().pnce_server_add_pilot(self._s, pl.handle), "pnce_server_add_pilot")
            self._pilots[N] = pl
        return self._pilots[N]

    def prepare(self, Ns, caps=CAPACITIES[:3]):
        """Capture the graphs of every (N, lag class) bucket of the given PN lengths, for
        every slot and capacity, before serving starts."""
        with torch.cuda.device(self.device):
            for N in Ns:
                self.pilot(N)
                for klc in sorted({kl_class(k, N) for k in KL_CLASSES if k <= N} | {kl_class(N, N)}):
                    for c in caps:
                        check(lib().pnce_server_prepare(self._s, N, klc, c),
                              "pnce_server_prepare")

    def run(self, requests: list) -> dict:
        for N in {r.N for r in requests}:
            self.pilot(N)
        reqs = _req_table(requests)
        out = np.zeros(len(requests), dtype=OUT_DTYPE)
        out["batch"] = -1
        out["status"] = -1                              # not run (the call fills it in)
        nb = C.c_int(0)
        with torch.cuda.device(self.device):
            st = lib().pnce_server_run(self._s, reqs.ctypes.data, len(requests),
                                       out.ctypes.data, C.byref(nb))
        if st != _lib.PNCE_OK and np.all(out["status"] == -1):
            check(st, "pnce_server_run")                # refused before running anything
        stats = _native_stats(requests, out, nb.value)
        check(st, "pnce_server_run")                   # a status latched on the device
        return stats

    # -- online use: requests submitted as they come, results collected as they finish
    def start(self):
        """Begin a session (its clock starts now)."""
        check(lib().pnce_server_start(self._s), "pnce_server_start")

    def submit(self, r: Request) -> int:
        """Queue one request (arriving now); returns its ticket.  Its buffers must stay
        valid until poll() reports it."""
        self.pilot(r.N)
        q = _lib.ServeReq(r.y_addr, r.h_addr, r.M, r.N, r.K, r.L, 0.0)
        t = C.c_longlong(0)
        check(lib().pnce_server_submit(self._s, C.byref(q), C.byref(t)), "pnce_server_submit")
        return t.value

    def poll(self, max_out: int = 256) -> list:
        """One scheduling pass; [(ticket, result)] of up to max_out finished requests, each
        result an OUT_DTYPE record (times from the session start, batch, status)."""
        tickets = np.empty(max(1, max_out), dtype=np.int64)
        outs = np.empty(max(1, max_out), dtype=OUT_DTYPE)
        n = C.c_int(0)
        with torch.cuda.device(self.device):
            check(lib().pnce_server_poll(self._s, tickets.ctypes.data, outs.ctypes.data,
                                         max_out, C.byref(n)), "pnce_server_poll")
        return [(int(tickets[k]), outs[k]) for k in range(n.value)]

    def open_requests(self) -> int:
        """Requests of the session not yet reported by poll()."""
        n = C.c_int(0)
        check(lib().pnce_server_open(self._s, C.byref(n)), "pnce_server_open")
        return n.value

    def __del__(self):
        s = getattr(self, "_s", None)
        if s is not None and _lib._lib is not None:
            _lib._lib.pnce_server_destroy(s)
            self._s = None
