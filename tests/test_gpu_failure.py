"""Failure detection without a GPU fault: every device-side wait of the tensor-core kernel
is bounded.  With a test switch the per-stage pilot generator withholds one arrive, so the
MMA issuer's wait can never be satisfied; the kernel must give up after the wait limit,
latch PNCE_ETIMEOUT, drain its copies, free TMEM and return -- and the context must stay
usable for the next call."""
import numpy as np
import pytest
import torch

from oracle import pn_oracle as O
from synth import channel as C

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(monkeypatch):
    import paper_2206_05506_gb300 as pk
    dev = torch.device("cuda", 0)
    w = C.Workload("to", r=10, M=64, K=8, L=64, F=4, snr_db=(10.0,), seed=3)
    bits, _, Y = C.make(w)
    pilot = pk.Pilot(bits, device=dev)
    Yd = torch.from_numpy(Y).to(dev)
    assert pk.get_status(dev) == 0
    monkeypatch.setenv("PNCE_TC_STAGED_PILOT", "1")
    monkeypatch.setenv("PNCE_TC_TEST_DROP_ARRIVE", "1")
    monkeypatch.setenv("PNCE_WAIT_LIMIT_MS", "100")
    pk.estimate(Yd, pilot, w.K, w.L, dtype="fp16")
    assert pk.get_status(dev) == 5                    # PNCE_ETIMEOUT, latched and cleared
    monkeypatch.delenv("PNCE_TC_TEST_DROP_ARRIVE")
    H = pk.estimate(Yd, pilot, w.K, w.L, dtype="fp16")
    assert pk.get_status(dev) == 0
    assert O.nmse(H.cpu().numpy(), O.estimate(Y, bits, w.K, w.L)) <= 2e-3
