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
