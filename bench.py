"""Benchmark: PN-correlation channel estimation throughput on GB300.

One step = one pnce_estimate call over one batch: per-antenna quantisation of the
received blocks, then the tensor-core correlation with its epilogue, on synthetic
received blocks shaped like the precision workload (M=128 antennas, N=4095 m-sequence,
K=16 transmitters x L=128 taps, 512 frames, SNR 0/10/20/30 dB), inputs resident in
HBM.  The library's tracing records CUDA events around each kernel it
launches, on the stream the kernel runs on; the correlation kernels' durations give the
roofline figure.

value      CIR taps estimated per second (one tap = one complex H entry), all ranks
e2e        the same metric through pnce_estimate_host: host (pinned) Y in, host H out
roofline   the correlation kernel against the measured dense tensor peak for its dtype
cpu_baseline  the FP64 oracle (Toeplitz product through numpy's BLAS) on a frame sample

Multi-GPU: frames are independent, so every rank estimates its own batch with no
collective on the data path (weak scaling); NCCL is used for the timing barrier and the
max over ranks only.  --impl reference times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import channel as C  # noqa: E402

FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# dense tensor throughput of each operand type relative to bf16 (nominal GB300 figures)
DTYPE_RATIO = {"fp16": 1.0, "bf16": 1.0, "e4m3": 2.0, "tf32": 0.5}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return FALLBACK_PEAKS, "fallback"


def source_hash(text: str) -> str:
    """Hash of C/CUDA source with comments and whitespace removed."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    text = " ".join(text.split())
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def src_hash() -> str:
    """Hash of the tensor-core kernel source, so that a recorded ncu traffic figure stays
    valid across comment edits but not code edits."""
    with open(os.path.join(ROOT, "paper_2206_05506_gb300", "csrc", "pnce_tc.cu")) as fh:
        return source_hash(fh.read())


def traffic_from_profile(workload: str, dtype: str, frames: int):
    """DRAM bytes per launch of the correlation kernel from the committed ncu summary, or
    None when there is none for this kernel source / workload."""
    p = os.path.join(ROOT, "profiles", "tc_corr_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    e = d.get(f"{workload}:{dtype}")
    if not e or e.get("src_hash") != src_hash():
        return None
    # the capture may be of fewer frames: DRAM traffic scales with the frames processed
    return float(e["bytes_per_frame"]) * frames


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons; keeps the samples that arrive
    between mark_start() and mark_end() (plus one sampling period)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 50

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self, warm_s: float = 1.0):
        import threading

        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.lines.append((time.monotonic(), line))

        threading.Thread(target=reader, daemon=True).start()
        t_end = time.monotonic() + warm_s          # wait for the first samples to flow
        while not self.lines and time.monotonic() < t_end:
            time.sleep(0.01)

    def mark_start(self):
        self.t0 = time.monotonic()

    def mark_end(self):
        self.t1 = time.monotonic()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(self.PERIOD_MS / 1000.0 * 2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return self.summarize(list(self.lines), self.t0, self.t1 + self.PERIOD_MS / 1000.0)

    @staticmethod
    def summarize(lines, lo: float, hi: float):
        """Median SM clock, maximum clock, median power and the throttle reasons seen
        active among the (time, csv line) samples taken in [lo, hi]."""
        sm, mx, power, reasons = [], None, [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, line in lines:
            if not (lo <= t <= hi):
                continue
            r = [x.strip() for x in line.split(",")]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                power.append(float(r[3]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "samples": len(sm),
                "power_w_median": float(np.median(power)) if power else None,
                "reasons": sorted(reasons)}


def cpu_oracle_sample(bits, Y_sample, K, L, target_s=15.0, max_frames=None):
    """Time the FP64 oracle on a growing prefix of frames until about target_s of work."""
    from oracle import pn_oracle as O

    O.estimate(Y_sample[:1], bits, K, L)                      # warm (BLAS threads, caches)
    t0 = time.perf_counter()
    O.estimate(Y_sample[:2], bits, K, L)
    t1 = (time.perf_counter() - t0) / 2
    nf = int(max(1, min(Y_sample.shape[0], (max_frames or 10 ** 9), round(target_s / max(t1, 1e-3)))))
    t0 = time.perf_counter()
    H = O.estimate(Y_sample[:nf], bits, K, L)
    dt = time.perf_counter() - t0
    return nf, dt, H


def _nmse(est, ref) -> float:
    est = np.asarray(est).astype(np.complex128)
    ref = np.asarray(ref).astype(np.complex128)
    return float(np.sum(np.abs(est - ref) ** 2) / np.sum(np.abs(ref) ** 2))


def nmse_stats(est, ref, frame_snr, chunk: int = 32) -> dict:
    """NMSE of est against the oracle's ref (both [F, ...]) over all frames, per SNR of the
    sweep (frame f at frame_snr[f]) and the worst frame."""
    est = np.asarray(est)
    nf = ref.shape[0]
    num = np.empty(nf)
    den = np.empty(nf)
    for f0 in range(0, nf, chunk):
        e = est[f0:f0 + chunk].astype(np.complex128)
        r = np.asarray(ref[f0:f0 + chunk]).astype(np.complex128)
        ax = tuple(range(1, e.ndim))
        num[f0:f0 + chunk] = (np.abs(e - r) ** 2).sum(axis=ax)
        den[f0:f0 + chunk] = (np.abs(r) ** 2).sum(axis=ax)
    snr = np.asarray(frame_snr)[:nf]
    return {"nmse": float(num.sum() / den.sum()),
            "nmse_by_snr_db": {f"{s:g}": float(num[snr == s].sum() / den[snr == s].sum())
                               for s in np.unique(snr)},
            "nmse_worst_frame": float(np.max(num / den)), "frames": int(nf)}


# Received blocks of the serving trace: 32 per (M, N) shape, 471 MB in all (3.6x L2), handed
# to the requests of each shape in turn, so that a request's block was last read about 512
# requests (~470 MB of other blocks) earlier and comes over the host link, not from L2.
SERVING_SLOTS = 32


def serving_payloads():
    from synth import serving as S
    return S.payload_pool(slots=SERVING_SLOTS, seed=0)


def oracle_references() -> dict:
    """Part of the cpu_baseline leg: the oracle's results that the serving spot check and
    the small-case leg compare with.  serving: for every payload of the serving pool, its
    estimate at all N lags (a request's expected result is the first K*L of them); small:
    the one-frame launch-latency case."""
    from oracle import pn_oracle as O
    from synth import serving as S

    full = {}
    for (M, N), Yp in serving_payloads().items():
        bits = S.pilot_bits(N)
        for slot in range(Yp.shape[0]):
            full[(M, N, slot)] = O.estimate(Yp[[slot]], bits, 1, N)[0, :, 0, :]
    w = C.SMALL
    bits, _, Y = C.make(w)
    ps = C.PAPER_SCALE
    pbits, _, pY = C.make(ps)
    return {"serving": full, "small": O.estimate(Y, bits, w.K, w.L),
            "paper_scale": O.estimate(pY, pbits, ps.K, ps.L)}


SWEEP_RATES_HZ = (10000.0, 20000.0, 40000.0, 80000.0, 120000.0, 160000.0)
# batches in flight (one stream each): 8 against 4 cut the fp16 p99 at 120k frames/s from
# 1.2 to 0.28 ms; the GPU time of a batch is mostly host-link latency, which overlaps
SERVING_STREAMS = 8


def knee_of(sweep: list):
    """The highest offered rate (rows in increasing order) still delivered (>= 95 %) with
    p99 within 4x of the lowest rate's, or None."""
    if not sweep:
        return None
    base_p99 = sweep[0]["p99_ms"]
    knee = None
    for row in sweep:
        if row["delivered_frames_per_s"] >= 0.95 * row["offered_hz"] and \
                row["p99_ms"] <= 4.0 * base_p99:
            knee = row["offered_hz"]
    return knee


def run_serving(dev, seconds: float, rate_hz: float = 20000.0, refs=None,
                sweep_rates=SWEEP_RATES_HZ, sweep_seconds: float = 2.0):
    """Poisson request stream (uneven M, N, K, L) through the continuous-batching server,
    tensor cores (fp16) and the plain FP32 SIMT path on the same trace, each through the
    library's native serving loop (the reported figures) and through the Python loop with
    the same rules (`python_loop`).  refs: the oracle's results per payload (from
    oracle_references) for the spot check, or None.  Then, per path and loop, an
    arrival-rate sweep (shorter traces): p50 / p99 latency and delivered frames/s at each
    offered rate, and the knee -- the highest offered rate still delivered (>= 95 %) with
    p99 within 4x of the lowest rate's."""
    import torch

    from paper_2206_05506_gb300 import serve
    from synth import serving as S

    pool = serving_payloads()
    pinned = {k: torch.from_numpy(v).pin_memory() for k, v in pool.items()}
    ring_elems = 64 << 20                      # 512 MB of page-locked results, reused in turn

    def trace(rate, secs, seed):
        specs = S.poisson_trace(rate, secs, seed=seed, payload_slots=SERVING_SLOTS)
        turn = {}
        for sp in specs:                       # each shape's blocks in turn (see SERVING_SLOTS)
            sp.slot = turn.get((sp.M, sp.N), 0)
            turn[(sp.M, sp.N)] = (sp.slot + 1) % SERVING_SLOTS
        return specs

    specs = trace(rate_hz, seconds, 0)
    ring = torch.zeros(ring_elems, dtype=torch.complex64, pin_memory=True)
    # spot check: every 100th request keeps its result in a buffer of its own
    checked = [sp for sp in specs if sp.rid % 100 == 0]
    check_buf = torch.zeros(max(1, sum(sp.M * sp.K * sp.L for sp in checked)),
                            dtype=torch.complex64, pin_memory=True)

    def requests(specs, spot):
        reqs, off, coff = [], 0, 0
        for sp in specs:
            n = sp.M * sp.K * sp.L
            y = pinned[(sp.M, sp.N)]
            y_addr = y.data_ptr() + sp.slot * sp.M * sp.N * 8
            if spot and sp.rid % 100 == 0:
                r = serve.Request(sp.rid, sp.t_arrival, sp.M, sp.N, sp.K, sp.L, y_addr,
                                  check_buf.data_ptr() + coff * 8)
                r.coff = coff
                coff += n
            else:
                if off + n > ring_elems:
                    off = 0
                r = serve.Request(sp.rid, sp.t_arrival, sp.M, sp.N, sp.K, sp.L, y_addr,
                                  ring.data_ptr() + off * 8)
                off += n
            reqs.append(r)
        return reqs

    res = {"rate_hz": rate_hz, "seconds": seconds, "requests": len(specs)}
    sweep_specs = {rate: trace(rate, sweep_seconds, 1 + i) for i, rate in enumerate(sweep_rates)}
    def measure(run):
        """The main trace (with the oracle spot check) and the rate sweep through `run`."""
        reqs = requests(specs, True)
        run([serve.Request(-1, 0.0, r.M, r.N, r.K, r.L, r.y_addr, r.h_addr)
             for r in reqs[:200]])                          # warm the path
        st = run(reqs)
        # accuracy of the sampled requests against the oracle's results
        errs = []
        for r in reqs if refs is not None else []:
            if r.rid % 100:
                continue
            n = r.M * r.K * r.L
            H = check_buf[r.coff:r.coff + n].numpy().reshape(r.M, r.K * r.L)
            want = refs[(r.M, r.N, specs[r.rid].slot)][:, :r.K * r.L]
            errs.append(_nmse(H, want))
        st["spot_check"] = {"requests": len(errs), "share": len(errs) / max(1, len(reqs)),
                            "nmse_max": float(max(errs)) if errs else None,
                            "nmse_median": float(np.median(errs)) if errs else None}
        sweep = []
        for rate in sweep_rates:
            sst = run(requests(sweep_specs[rate], False))
            sweep.append({"offered_hz": rate, "delivered_frames_per_s": sst["frames_per_s"],
                          "p50_ms": sst["p50_ms"], "p99_ms": sst["p99_ms"],
                          "max_ms": sst["max_ms"], "mean_batch_rows": sst["mean_batch_rows"],
                          "failed": sst["failed"]})
        st["rate_sweep"] = {"seconds_per_rate": sweep_seconds, "rows": sweep,
                            "knee_offered_hz": knee_of(sweep)}
        return st

    res["loop"] = ("native: the scheduling loop in the library (pnce_server_run); "
                   "python_loop: the same rules in serve.Server")
    for dtype, name in (("fp16", "fp16_tensor_core"), ("fp32", "fp32_simt")):
        nat = serve.NativeServer(S.pilot_bits, device=dev, dtype=dtype, slots=SERVING_STREAMS,
                                 mem_cap_bytes=40e9)
        nat.prepare([255, 511, 1023, 2047], caps=serve.CAPACITIES)
        st = measure(nat.run)
        del nat
        eng = serve.GpuEngine(S.pilot_bits, device=dev, dtype=dtype, slots=SERVING_STREAMS)
        eng.prepare([255, 511, 1023, 2047], caps=serve.CAPACITIES)
        st["python_loop"] = measure(lambda rq: serve.Server(eng, mem_cap_bytes=40e9).run(rq))
        res[name] = st
        del eng
        torch.cuda.empty_cache()
    return res


# One-request serving batches: (M, N, K, L) of a large and a small request
SERVING_BATCH_CASES = ((256, 1023, 1, 1023), (64, 511, 4, 32))


def run_serving_batch(dev, replays: int):
    """GPU time of one serving batch holding a single request, per path (fp16 tensor
    cores, FP32 SIMT) and request shape: a one-stream engine replays the batch's captured
    graph (prep, gather + quantise or gather, correlation, scatter), each replay reading a
    different page-locked block from a pool larger than L2 and writing its result to
    page-locked memory; CUDA events around each replay, median and 90th percentile.  Then
    the correlation kernel alone (traced eager runs) against its roofline."""
    import torch

    import paper_2206_05506_gb300 as pk
    from paper_2206_05506_gb300 import serve
    from synth import serving as S

    out = {}
    gen = torch.Generator().manual_seed(0)
    for M, N, K, L in SERVING_BATCH_CASES:
        blocks = max(2, (320 << 20) // (M * N * 8))          # 320 MB of received blocks
        pool = torch.randn((blocks, M, N), dtype=torch.complex64, generator=gen).pin_memory()
        H = torch.empty((M, K * L), dtype=torch.complex64).pin_memory()
        for dtype in ("fp16", "fp32"):
            eng = serve.GpuEngine(S.pilot_bits, device=dev, dtype=dtype, slots=1)
            cap = next(c for c in serve.CAPACITIES if c >= M)
            shape = eng._shape(0, N, serve.kl_class(K * L, N), cap)
            s = eng.streams[0]
            ts = []
            for i in range(replays + 20):
                req = [serve.Request(0, 0.0, M, N, K, L, pool[i % blocks].data_ptr(),
                                     H.data_ptr())]
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(s)
                shape.run(eng, 0, req)
                e1.record(s)
                e1.synchronize()
                if i >= 20:
                    ts.append(e0.elapsed_time(e1) * 1e3)
            # the correlation kernel's own time: eager runs of the same batch with the
            # library's tracing on (no dependent-launch overlap, so the kernel is alone)
            graph, shape.graph = shape.graph, None
            pk.trace_enable(True, dev)
            pk.trace_read(dev)
            for i in range(20):
                shape.run(eng, 0, [serve.Request(0, 0.0, M, N, K, L,
                                                 pool[i % blocks].data_ptr(), H.data_ptr())])
            torch.cuda.synchronize()
            kind = "correlate" if dtype != "fp32" else "simt"
            kt = [t for k, t in pk.trace_read(dev) if k == kind]
            pk.trace_enable(False, dev)
            shape.graph = graph
            kern_us = float(np.median(kt)) * 1e3 if kt else None
            flops = 4.0 * N * M * K * L                          # the request's own taps
            peaks, _ = load_peaks()
            row = {"gpu_us_median": float(np.median(ts)),
                   "gpu_us_p90": float(np.percentile(ts, 90)), "replays": replays,
                   "bytes_in": M * N * 8, "bytes_out": M * K * L * 8,
                   "correlation_kernel_us": kern_us}
            if kern_us:
                achieved = flops / (kern_us * 1e-6) / 1e12
                sms = torch.cuda.get_device_properties(dev).multi_processor_count
                peak = (peaks["bf16_tflops"] * DTYPE_RATIO[dtype] if dtype != "fp32"
                        else sms * 128 * 2 * 2070e6 / 1e12)
                row["correlation_roofline"] = {
                    "bound": "tensor" if dtype != "fp32" else "alu", "achieved": achieved,
                    "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "note": "a lone request: a few CTAs, bound by set-up and drain latency"}
            out[f"{dtype}_m{M}_n{N}_kl{K * L}"] = row
            del eng
        del pool
    return out


def run_paper_scale(dev, ref=None, reps: int = 50):
    """The paper-scale workload (M = 64, N = 1023, K = 8, L = 64, 128 frames, SNR 0/10/20
    dB): the plain FP32 SIMT path against the TF32 tensor-core path (and fp16), each with
    its step time, throughput, the roofline fraction of its correlation kernel and, given
    the oracle's estimate `ref`, its NMSE overall and per SNR."""
    import torch

    import paper_2206_05506_gb300 as pk

    w = C.PAPER_SCALE
    bits, _, Y = C.make(w)
    Yd = torch.from_numpy(Y).to(dev)
    pilot = pk.Pilot(bits, device=dev)
    H = torch.empty((w.F, w.M, w.K, w.L), dtype=torch.complex64, device=dev)
    peaks, peak_src = load_peaks()
    taps = w.F * w.M * w.K * w.L
    flops = 4.0 * w.F * w.M * w.N * w.K * w.L
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = torch.cuda.current_stream(dev)
    out = {"workload": w.name}
    for dt in ("fp32", "tf32", "fp16"):
        ws = (torch.empty(pk.workspace_size(w.F, w.M, w.N, w.K, w.L, dt), dtype=torch.uint8,
                          device=dev) if dt != "fp32" else None)
        for _ in range(5):
            pk.estimate(Yd, pilot, w.K, w.L, dtype=dt, out=H, workspace=ws)
        torch.cuda.synchronize()
        pk.trace_enable(True, dev)
        pk.trace_read(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            pk.estimate(Yd, pilot, w.K, w.L, dtype=dt, out=H, workspace=ws)
        e1.record(stream)
        torch.cuda.synchronize()
        tr = pk.trace_read(dev)
        pk.trace_enable(False, dev)
        ms = e0.elapsed_time(e1) / reps
        kind = "simt" if dt == "fp32" else "correlate"
        kern_ms = float(np.median([t for k, t in tr if k == kind]))
        q_ms = [t for k, t in tr if k == "quantize"]
        achieved = flops / (kern_ms / 1e3) / 1e12
        if dt == "fp32":
            peak = sms * 128 * 2 * 2070.0 * 1e6 / 1e12
            roof = {"bound": "alu", "kernel": "simt_corr_kernel", "achieved": achieved,
                    "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 flop x 2070 MHz"}
        else:
            peak = peaks["bf16_tflops"] * DTYPE_RATIO[dt]
            roof = {"bound": "tensor", "kernel": "tc_corr_kernel", "achieved": achieved,
                    "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "peak_source": f"{peak_src} burst bf16 x {DTYPE_RATIO[dt]}"}
        row = {"ms_per_step": ms, "value": taps / (ms / 1e3), "unit": "taps/s",
               "kernel_ms": kern_ms,
               "quantize_ms": float(np.median(q_ms)) if q_ms else 0.0, "roofline": roof}
        if ref is not None:
            row.update(nmse_stats(H.cpu().numpy(), ref, w.frame_snr()))
        out[dt] = row
        del ws
    assert pk.get_status(dev) == 0
    return out


def rank_first_frame(F: int, rank: int, world: int) -> int:
    """Weak scaling: every rank estimates its own batch of F frames, rank r taking frames
    [r*F, (r+1)*F) of the synthetic stream (no data crosses ranks)."""
    return rank * F if world > 1 else 0


def max_over_ranks(ms: float, world: int, device=None) -> float:
    """The slowest rank's time (the whole job finishes with it)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_yardsticks(dev, bits, Y, pilot, K, L, taps_per_step, reps: int = 20):
    """O(N log N) alternatives on the same batch, for comparison only (not the paper's
    method): the library's fast m-sequence transform (permutation + Walsh-Hadamard, FP32,
    HBM-bound: 8 B read per sample, 8 B written per lag) and a cuFFT circular correlation
    through torch.fft.  Each reports ms per batch and its NMSE against the library's FP32
    SIMT estimate of the same batch."""
    import torch

    import paper_2206_05506_gb300 as pk
    F, M, N = Y.shape
    KL = K * L
    peaks, _ = load_peaks()
    out = {}
    H32 = pk.estimate(Y, pilot, K, L, dtype="fp32")

    def nmse(a):
        return float(((a - H32).abs() ** 2).sum().item() / (H32.abs() ** 2).sum().item())

    fmt = pk.FmtPilot(bits, device=dev)
    Hf = torch.empty_like(H32)
    pk.trace_enable(True, dev)
    for _ in range(3):
        pk.estimate_fmt(Y, fmt, K, L, out=Hf)
    pk.trace_read(dev)
    for _ in range(reps):
        pk.estimate_fmt(Y, fmt, K, L, out=Hf)
    ms = float(np.median([t for kind, t in pk.trace_read(dev) if kind == "fmt"]))
    pk.trace_enable(False, dev)
    gbs = (F * M * (8.0 * N + 8.0 * KL)) / (ms / 1e3) / 1e9
    out["fast_msequence_transform"] = {
        "ms_per_batch": ms, "value": taps_per_step / (ms / 1e3), "unit": "taps/s",
        "achieved_gbs": gbs, "hbm_peak_gbs": peaks["hbm_gbs"],
        "frac_hbm": gbs / peaks["hbm_gbs"], "nmse_vs_fp32_simt": nmse(Hf)}
    del Hf, fmt
    # cuFFT: H = ifft(fft(y) * conj(fft(p)))[:KL] / N, through torch (library FFTs)
    p = torch.from_numpy(1.0 - 2.0 * bits.astype(np.float32)).to(dev)
    Pc = torch.conj(torch.fft.fft(p.to(torch.complex64)))

    def fft_corr():
        c = torch.fft.ifft(torch.fft.fft(Y, dim=-1) * Pc, dim=-1)
        return c[..., :KL]

    for _ in range(2):
        Hc = fft_corr()
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record()
    n = 5
    for _ in range(n):
        Hc = fft_corr()
    a1.record()
    torch.cuda.synchronize()
    ms = a0.elapsed_time(a1) / n
    Hc = Hc.reshape(H32.shape) / N
    out["cufft_circular_correlation"] = {
        "ms_per_batch": ms, "value": taps_per_step / (ms / 1e3), "unit": "taps/s",
        "nmse_vs_fp32_simt": nmse(Hc),
        "note": "torch.fft (cuFFT) forward + inverse over all N lags, then the first K*L"}
    del Hc, Pc, H32
    torch.cuda.empty_cache()
    return out


def run_layouts(dev, pilot, Y, K, L, taps_per_step, reps: int = 30):
    """The pilot-slot layouts on the same batch (fp16): rows with an L-sample cyclic prefix
    in front (the prefix repeats the block's tail), and the even-spread shift rule
    k * floor(N / K) of Eq. 8.  ms per step beside the plain step's."""
    import torch

    import paper_2206_05506_gb300 as pk

    F, M, N = Y.shape
    Ycp = torch.empty((F, M, N + L), dtype=torch.complex64, device=dev)
    Ycp[:, :, L:] = Y
    Ycp[:, :, :L] = Y[:, :, N - L:]
    H = torch.empty((F, M, K, L), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)
    out = {}
    for name, src, kw in (("cyclic_prefix", Ycp, {"cp_len": L}),
                          ("spread_shifts", Y, {"shift_rule": "spread"})):
        for _ in range(3):
            pk.estimate(src, pilot, K, L, dtype="fp16", out=H, **kw)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            pk.estimate(src, pilot, K, L, dtype="fp16", out=H, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms_per_step": ms, "value": taps_per_step / (ms / 1e3)}
    del Ycp
    assert pk.get_status(dev) == 0
    return out


def run_small_case(dev, ref=None, calls: int = 200):
    """Launch-latency case: one frame of 8 antennas, N = 127, K = 2, L = 16 (8 KB in, 2 KB
    out), FP32 (the few-lags SIMT kernel).  Per call: the kernel's device time (the
    library's trace events around the launch), the host wall time of the call and its
    synchronisation, and end to end from page-locked host memory (pnce_estimate_host: copy
    in, estimate, copy out).  ref: the oracle's result (from oracle_references) or None."""
    import torch

    import paper_2206_05506_gb300 as pk

    w = C.SMALL
    bits, _, Y = C.make(w)
    Yd = torch.from_numpy(Y).to(dev)
    pilot = pk.Pilot(bits, device=dev)
    H = torch.empty((w.F, w.M, w.K, w.L), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(20):
        pk.estimate(Yd, pilot, w.K, w.L, dtype="fp32", out=H)
    torch.cuda.synchronize()
    call_us = []
    pk.trace_enable(True, dev)
    pk.trace_read(dev)
    for _ in range(calls):
        t0 = time.perf_counter()
        pk.estimate(Yd, pilot, w.K, w.L, dtype="fp32", out=H)
        stream.synchronize()
        call_us.append((time.perf_counter() - t0) * 1e6)
    dev_us = [t * 1e3 for kind, t in pk.trace_read(dev) if kind == "simt"]
    pk.trace_enable(False, dev)
    Yh = torch.from_numpy(Y).pin_memory()
    Hh = torch.empty((w.F, w.M, w.K, w.L), dtype=torch.complex64).pin_memory()
    for _ in range(20):
        pk.estimate_host(Yh, pilot, w.K, w.L, dtype="fp32", out=Hh)
    e2e_us = []
    for _ in range(calls):
        t0 = time.perf_counter()
        pk.estimate_host(Yh, pilot, w.K, w.L, dtype="fp32", out=Hh)
        e2e_us.append((time.perf_counter() - t0) * 1e6)
    out = {"workload": w.name, "dtype": "fp32", "calls": calls,
           "kernel_us_median": float(np.median(dev_us)),
           "call_us_median": float(np.median(call_us)),
           "e2e_host_us_median": float(np.median(e2e_us)),
           "e2e_host_us_p99": float(np.percentile(e2e_us, 99)),
           "taps": w.F * w.M * w.K * w.L,
           "e2e_matches_device_result": bool(torch.equal(Hh, H.cpu()))}
    if ref is not None:
        out["nmse_vs_oracle"] = _nmse(H.cpu().numpy(), ref)
    return out


def run_differentiation(dev, steps: int = 20):
    """Relaxed-pilot forward + adjoint (dLoss/dY and dLoss/dtheta) on the differentiation
    workload (M=64, N=1023, K=8, L=64, 64 frames, FP32), as one training step would."""
    import torch

    import paper_2206_05506_gb300 as pk
    from paper_2206_05506_gb300.autograd import relaxed_estimate

    w = C.DIFFERENTIATION
    bits, h, Y = C.make(w)
    Yd = torch.from_numpy(Y).to(dev).requires_grad_(True)
    Ht = torch.from_numpy(h.astype(np.complex64)).to(dev)
    theta = torch.randn(w.N, device=dev, generator=torch.Generator(dev).manual_seed(0))
    theta.requires_grad_(True)

    def step():
        Yd.grad = None
        theta.grad = None
        loss = (relaxed_estimate(Yd, theta, w.K, w.L) - Ht).abs().pow(2).mean()
        loss.backward()
        return loss

    for _ in range(3):
        step()
    pk.trace_enable(True, dev)
    pk.trace_read(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    pk.trace_enable(False, dev)
    ms = e0.elapsed_time(e1) / steps
    fl = 4.0 * w.F * w.M * w.N * w.K * w.L          # one correlation-sized pass
    return {"workload": w.name, "ms_per_step": ms,
            "forward_plus_adjoint_tflops": 3 * fl / (ms / 1e3) / 1e12,
            "note": "loss and its torch elementwise ops included; 3 correlation-sized passes"}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args, w):
    """FP64 CPU oracle as the reference arm: each step estimates a bounded frame sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import pn_oracle as O

    nf = args.ref_frames
    bits, Y = C.make_received(w, frames=nf)
    for _ in range(args.warmup):
        O.estimate(Y, bits, w.K, w.L)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.estimate(Y, bits, w.K, w.L)
    dt = time.perf_counter() - t0
    taps = nf * w.M * w.K * w.L
    value = taps * args.steps / dt
    line = {
        "impl": "reference", "metric": "CIR taps estimated/s", "value": value, "unit": "taps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "frames_per_step": nf, "M": w.M, "N": w.N, "K": w.K,
                   "L": w.L},
        "cpu_baseline": {"value": value, "unit": "taps/s", "cores": host_cores(),
                         "kind": "oracle",
                         "sample": f"{nf} of {w.F} frames per step, FP64 Toeplitz product"},
        "e2e": {"value": value, "unit": "taps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=C.PRECISION.name, choices=sorted(C.WORKLOADS))
    ap.add_argument("--dtype", default="fp16", choices=["fp32", "tf32", "fp16", "bf16", "e4m3"])
    ap.add_argument("--frames", type=int, default=None, help="override frames per step")
    ap.add_argument("--K", type=int, default=None, help="override the transmitters (K)")
    ap.add_argument("--L", type=int, default=None, help="override the taps per transmitter (L)")
    ap.add_argument("--e2e-steps", type=int, default=16)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--ref-frames", type=int, default=8, help="frames per reference step")
    ap.add_argument("--serving-seconds", type=float, default=10.0,
                    help="length of the Poisson serving trace (0: skip)")
    ap.add_argument("--serving-sweep", type=int, default=1,
                    help="also sweep the offered rate of the serving trace (1/0)")
    ap.add_argument("--serving-batch-replays", type=int, default=300,
                    help="replays per case of a one-request serving batch (0: skip)")
    ap.add_argument("--differentiation", type=int, default=1,
                    help="also time the relaxed-pilot forward + adjoint (1/0)")
    ap.add_argument("--yardsticks", type=int, default=1,
                    help="time the O(N log N) yardsticks (fast m-sequence transform, cuFFT)")
    ap.add_argument("--layouts", type=int, default=1,
                    help="time the cyclic-prefix and even-spread pilot layouts (1/0)")
    ap.add_argument("--small-case", type=int, default=1,
                    help="time the one-frame launch-latency case (1/0)")
    ap.add_argument("--other-dtypes", type=int, default=1,
                    help="also time the other arithmetics on the same batch (1/0)")
    ap.add_argument("--paper-experiments", type=int, default=10,
                    help="iterations per point of the Sec. IV experiments (0: skip)")
    ap.add_argument("--paper-scale", type=int, default=1,
                    help="time FP32 SIMT vs TF32 / fp16 on the paper-scale workload (1/0)")
    args = ap.parse_args()

    w = C.WORKLOADS[args.workload]
    if args.frames or args.K or args.L:
        F = args.frames or w.F
        K = args.K or w.K
        L = args.L or w.L
        name = w.name if (F, K, L) == (w.F, w.K, w.L) else f"n{w.N}_m{w.M}_k{K}_l{L}_f{F}"
        w = C.Workload(name, r=w.r, M=w.M, K=K, L=L, F=F, snr_db=w.snr_db, seed=w.seed)
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    import torch.distributed as dist

    import paper_2206_05506_gb300 as pk

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- inputs (each rank its own batch: frames offset by rank)
    bits, Y_host = C.make_received(w, first=rank_first_frame(w.F, rank, world))
    Y_pin = torch.from_numpy(Y_host).pin_memory()
    Y = Y_pin.to(dev)
    F, M, N, K, L = w.F, w.M, w.N, w.K, w.L
    dt = args.dtype
    pilot = pk.Pilot(bits, device=dev)
    H = torch.empty((F, M, K, L), dtype=torch.complex64, device=dev)
    ws = None
    if dt != "fp32":
        ws = torch.empty(pk.workspace_size(F, M, N, K, L, dt), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        # the product call (quantise, then correlate; PNCE_OVERLAP_CHUNKS would overlap them)
        pk.estimate(Y, pilot, K, L, dtype=dt, out=H, workspace=ws)

    pk.trace_enable(True, dev)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert pk.get_status(dev) == 0
    pk.trace_read(dev)

    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    clocks.mark_start()
    e_start.record(stream)
    for i in range(args.steps):
        step()
    e_end.record(stream)
    torch.cuda.synchronize()
    clocks.mark_end()
    barrier()
    clk = clocks.stop()
    trace = pk.trace_read(dev)       # (kind, ms) of every kernel launched in the timed region
    pk.trace_enable(False, dev)
    total_ms = max_over_ranks(e_start.elapsed_time(e_end), world, dev)
    assert pk.get_status(dev) == 0
    main_kind = "simt" if dt == "fp32" else "correlate"
    corr_ms = [ms for kind, ms in trace if kind == main_kind]
    quant_ms = [ms for kind, ms in trace if kind == "quantize"]
    launches = len(trace)
    nch = max(1, len(corr_ms) // args.steps)

    taps_per_step = F * M * K * L
    value = taps_per_step * args.steps * world / (total_ms / 1e3)

    # the correlation kernel alone (operand quantised once, nothing running beside it), for
    # comparison with its in-step duration above
    alone_ms = None
    if dt != "fp32":
        q = pk.quantize(Y, dt, workspace=ws)
        for _ in range(3):
            pk.correlate_quantized(ws, pilot, F, M, K, L, dt, out=H)
        pk.trace_enable(True, dev)
        pk.trace_read(dev)
        for _ in range(20):
            pk.correlate_quantized(ws, pilot, F, M, K, L, dt, out=H)
        alone_ms = float(np.mean([ms for _, ms in pk.trace_read(dev)]))
        pk.trace_enable(False, dev)
        del q

    # ---- end to end through the host-buffer entry point
    H_pin = torch.empty((F, M, K, L), dtype=torch.complex64, pin_memory=True)
    hws = torch.empty(pk.host_workspace_size(F, M, N, K, L, dt), dtype=torch.uint8, device=dev)
    pk.estimate_host(Y_pin, pilot, K, L, dtype=dt, out=H_pin, workspace=hws)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    per_step = []
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.e2e_steps):
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        pk.lib().pnce_estimate_host(pilot.ctx.handle, pilot.handle, Y_pin.data_ptr(), F, M, N, K,
                                    L, pk.DTYPES[dt], hws.data_ptr(), hws.numel(),
                                    H_pin.data_ptr(), stream.cuda_stream)
        s1.record(stream)
        per_step.append((s0, s1))
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    e2e_med_ms = max_over_ranks(float(np.median([a.elapsed_time(b) for a, b in per_step])), world, dev)
    e2e_value = taps_per_step * args.e2e_steps * world / (e2e_ms / 1e3)
    assert pk.get_status(dev) == 0
    e2e_matches = bool(torch.equal(H_pin, H.cpu()))

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    # ---- roofline of the correlation kernel
    peaks, peak_src = load_peaks()
    # per correlation launch (one frame chunk): real GEMM of 2 Fc M rows x N x KL, 2 flop
    # per MAC (the SIMT path does the same 2 FMA per complex sample and lag)
    flops = 4.0 * (F / nch) * M * N * K * L
    kern_ms = float(np.mean(corr_ms))
    if dt == "fp32":
        # FP32 CUDA-core peak: 152 SMs x 128 FMA lanes x 2 flop x SM clock (2070 MHz max)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = (clk or {}).get("sm_mhz") or 2070.0
        peak = sms * 128 * 2 * mhz * 1e6 / 1e12
        achieved = flops / (kern_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": "simt_corr_kernel",
                "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz"}
    else:
        long_region = total_ms > 1000.0
        base = peaks["bf16_tflops_sustained" if long_region else "bf16_tflops"]
        peak = base * DTYPE_RATIO[dt]
        achieved = flops / (kern_ms / 1e3) / 1e12
        alone = 4.0 * F * M * N * K * L / (alone_ms / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "kernel_alone": {"ms_per_launch": alone_ms, "frames_per_launch": F,
                                 "achieved": alone, "frac": alone / peak},
                "traffic": traffic_from_profile(w.name, dt, F / nch),
                "kernel": "tc_corr_kernel", "peak_source":
                f"{peak_src} {'sustained' if long_region else 'burst'} bf16 x {DTYPE_RATIO[dt]}"}

    # ---- CPU baseline (FP64 oracle) on a frame sample, plus accuracy of those frames.  It
    # and the legs below describe the single-GPU configuration: they run at N = 1 only
    # (with N > 1 they would keep every GPU of the job idle for minutes).
    single = world == 1
    cpu = None
    nmse = None
    accuracy = None
    if not args.no_cpu and single:
        from oracle import pn_oracle as O
        nf, cdt, Href = cpu_oracle_sample(bits, Y_host, K, L)
        cpu = {"value": nf * M * K * L / cdt, "unit": "taps/s", "cores": host_cores(),
               "kind": "oracle",
               "sample": f"first {nf} of {F} frames, FP64 Toeplitz product (numpy BLAS)"}
        accuracy = nmse_stats(H[:nf].cpu().numpy(), Href, w.frame_snr())
        nmse = accuracy["nmse"]
        refs = oracle_references()
    else:
        refs = {}
        Href = None

    serving = (run_serving(dev, args.serving_seconds, refs=refs.get("serving"),
                           sweep_rates=SWEEP_RATES_HZ if args.serving_sweep else ())
               if args.serving_seconds > 0 and single else None)
    serving_batch = (run_serving_batch(dev, args.serving_batch_replays)
                     if args.serving_batch_replays > 0 and single else None)
    small = run_small_case(dev, ref=refs.get("small")) if args.small_case and single else None
    differentiation = run_differentiation(dev) if args.differentiation and single else None

    # the other arithmetics on the same batch (shorter runs, same step definition)
    others = {}
    if args.other_dtypes and single:
        for odt in [d for d in ("e4m3", "bf16", "tf32", "fp16", "fp32") if d != dt]:
            ows = (torch.empty(pk.workspace_size(F, M, N, K, L, odt), dtype=torch.uint8,
                               device=dev) if odt != "fp32" else None)
            for _ in range(3):
                pk.estimate(Y, pilot, K, L, dtype=odt, out=H, workspace=ows)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            n_o = 50 if odt != "fp32" else 5
            a0.record(stream)
            for _ in range(n_o):
                pk.estimate(Y, pilot, K, L, dtype=odt, out=H, workspace=ows)
            a1.record(stream)
            torch.cuda.synchronize()
            ms_o = a0.elapsed_time(a1) / n_o
            others[odt] = {"ms_per_step": ms_o, "value": taps_per_step / (ms_o / 1e3)}
            if Href is not None:           # the same frames the oracle estimated
                others[odt].update(nmse_stats(H[:Href.shape[0]].cpu().numpy(), Href,
                                              w.frame_snr()))
            del ows
        assert pk.get_status(dev) == 0

    paper_scale = (run_paper_scale(dev, refs.get("paper_scale"))
                   if args.paper_scale and single else None)
    paper_exp = None
    if args.paper_experiments > 0 and single:
        import paper_experiments as PE
        paper_exp = PE.run(pk, dev, "fp16", iters=args.paper_experiments)
        paper_exp["claims"] = PE.claims(paper_exp)
    yard = (run_yardsticks(dev, bits, Y, pilot, K, L, taps_per_step)
            if args.yardsticks and single else None)
    layouts = (run_layouts(dev, pilot, Y, K, L, taps_per_step)
               if args.layouts and dt == "fp16" and single else None)

    line = {
        "metric": "CIR taps estimated/s", "value": value, "unit": "taps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dt,
        "data": "synthetic",
        "config": {"workload": w.name, "frames": F, "M": M, "N": N, "K": K, "L": L,
                   "snr_db": list(w.snr_db), "parallelism": f"frames x{world}",
                   "l2": f"inputs larger than L2 ({Y.numel() * 8 / 1e9:.2f} GB Y per step)"},
        "breakdown_ms": {"correlate_per_launch": kern_ms,
                         "correlate_launches_per_step": nch,
                         "quantize_per_launch": float(np.mean(quant_ms)) if quant_ms else 0.0,
                         "traced_kernels": launches},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": "taps/s",
                "h2d_bytes_per_step": int(Y_pin.numel() * 8),
                "d2h_bytes_per_step": int(H_pin.numel() * 8),
                "ms_per_step": e2e_ms / args.e2e_steps,
                "ms_per_step_median": e2e_med_ms,
                "value_from_median_step": taps_per_step * world / (e2e_med_ms / 1e3),
                "note": "copy-bound over the host link (~211 GB/s H2D measured); the host "
                        "is shared, so step times vary between runs",
                "matches_device_result": e2e_matches},
        "gpu_launches": launches,
        "clocks": clk,
        "nmse_vs_oracle": nmse,
        "accuracy": accuracy,
        "cpu_baseline": cpu,
        "serving": serving,
        "serving_batch": serving_batch,
        "small_case": small,
        "other_dtypes": others,
        "paper_scale": paper_scale,
        "paper_experiments": paper_exp,
        "differentiation": differentiation,
        "yardsticks": yard,
        "layouts": layouts,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
