"""Tracing: while enabled, every quantiser / correlation / adjoint launch of the entry
points is recorded (kind and event-timed milliseconds) in launch order; reading clears the
record; nothing is recorded while it is off."""
import numpy as np
import pytest
import torch

from synth import channel as C

pytestmark = pytest.mark.gpu


def test_trace_kinds_in_launch_order():
    import paper_2206_05506_gb300 as pk
    dev = torch.device("cuda", 0)
    w = C.Workload("tr", r=10, M=16, K=4, L=64, F=4, snr_db=(10.0,), seed=2)
    bits, _, Y = C.make(w)
    Yd = torch.from_numpy(Y).to(dev)
    pilot = pk.Pilot(bits, device=dev)
    fmt = pk.FmtPilot(bits, device=dev)
    theta = torch.randn(w.N, device=dev, generator=torch.Generator(dev).manual_seed(0))
    G = torch.randn(w.F, w.M, w.K, w.L, dtype=torch.complex64, device=dev)

    pk.estimate(Yd, pilot, w.K, w.L, dtype="fp16")          # warm every path untraced
    pk.trace_enable(True, dev)
    pk.trace_read(dev)
    pk.estimate(Yd, pilot, w.K, w.L, dtype="fp16")
    pk.estimate(Yd, pilot, w.K, w.L, dtype="fp32")
    pk.estimate_real_pilot(Yd, theta, w.K, w.L, pilot_map="tanh")
    pk.backward(theta, Yd, G, w.K, w.L, pilot_map="tanh")
    pk.estimate_fmt(Yd, fmt, w.K, w.L)
    rec = pk.trace_read(dev)
    assert [k for k, _ in rec] == ["quantize", "correlate", "simt", "simt", "adjoint", "fmt"]
    assert all(np.isfinite(t) and t > 0.0 for _, t in rec)
    assert pk.trace_read(dev) == []                          # the read cleared the record

    pk.trace_enable(False, dev)
    pk.estimate(Yd, pilot, w.K, w.L, dtype="fp16")
    assert pk.trace_read(dev) == []


def test_trace_covers_static_and_grouped_entry_points():
    # the allocation-free and the grouped (serving) entry points are traced like the others
    import ctypes as C_
    import paper_2206_05506_gb300 as pk
    from paper_2206_05506_gb300 import _lib
    dev = torch.device("cuda", 0)
    w = C.Workload("tr2", r=9, M=16, K=2, L=32, F=2, snr_db=(10.0,), seed=5)
    bits, _, Y = C.make(w)
    Yd = torch.from_numpy(Y).to(dev)
    pilot = pk.Pilot(bits, device=dev)
    H = torch.empty((w.F, w.M, w.K, w.L), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    # a grouped batch of one request (device buffers)
    desc = torch.zeros(C_.sizeof(_lib.ReqDesc), dtype=torch.uint8, pin_memory=True)
    d = (_lib.ReqDesc * 1).from_address(desc.data_ptr())
    Hg = torch.empty((w.M, w.K * w.L), dtype=torch.complex64, device=dev)
    d[0].Y, d[0].H, d[0].M, d[0].K, d[0].L, d[0].row_offset = \
        Yd[0].data_ptr(), Hg.data_ptr(), w.M, w.K, w.L, 0
    ws = torch.empty(pk.grouped_workspace_size(w.M, w.N, w.K * w.L, "fp16"), dtype=torch.uint8,
                     device=dev)
    for traced in (False, True):                     # warm untraced, then record
        pk.trace_enable(traced, dev)
        pk.trace_read(dev)
        assert pk.lib().pnce_estimate_static(pilot.ctx.handle, pilot.handle, Yd.data_ptr(), w.F,
                                             w.M, w.N, w.K, w.L, pk.DTYPES["fp16"],
                                             H.data_ptr(), stream) == 0
        pk.estimate_grouped(pilot, desc.data_ptr(), 1, w.M, w.K * w.L, "fp16", ws)
    rec = pk.trace_read(dev)
    pk.trace_enable(False, dev)
    assert [k for k, _ in rec] == ["quantize", "correlate", "quantize", "correlate"]
    assert all(np.isfinite(t) and t > 0.0 for _, t in rec)
    assert pk.get_status(dev) == 0
