"""The allocation-free entry point pnce_estimate_static, called through the C ABI.

It serves callers that cannot allocate device memory on their path (a real-time receive
chain that must not wait on the allocator, a host with a fixed memory budget): its
scratch is a fixed array inside the library.  Its results must match pnce_estimate, the
entry point that takes a caller-allocated workspace, call after call -- the array keeps
the previous call's contents, so two different inputs go through it back to back.

This file is collected last on purpose, and it must also pass on its own in a fresh
process.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import pn_oracle as O
from synth import channel as C_syn

pytestmark = pytest.mark.gpu

TOL_Q = {"fp16": 1e-9, "bf16": 1e-9, "tf32": 1e-9, "e4m3": 1e-6}
STATIC_BYTES = 64 << 20     # PNCE_STATIC_SCRATCH_BYTES in include/pnce.h


@pytest.fixture(scope="module")
def pk():
    import paper_2206_05506_gb300 as pk
    pk.lib()
    return pk


def _frames(w, first, frames):
    bits, Y = C_syn.make_received(w, frames=frames, first=first)
    return bits, Y


@pytest.mark.parametrize("dtype", ["fp16", "e4m3", "bf16", "tf32"])
def test_static_matches_workspace_entry_point_twice(pk, dtype):
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = C_syn.Workload("na", r=10, M=40, K=6, L=50, F=5, snr_db=(10.0,), seed=21)
    lib = pk.lib()
    dt = pk.DTYPES[dtype]
    bits, _ = _frames(w, 0, 1)
    pilot = pk.Pilot(bits, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    # two different inputs, back to back through the same scratch array
    for call, (first, frames) in enumerate([(0, 5), (5, 3)]):
        _, Y = _frames(w, first, frames)
        Yd = torch.from_numpy(Y).to(dev)
        F, M, N = Y.shape
        H_ref = pk.estimate(Yd, pilot, w.K, w.L, dtype=dtype)
        H = torch.full((F, M, w.K, w.L), complex(7.0, 7.0), dtype=torch.complex64, device=dev)
        st = lib.pnce_estimate_static(pilot.ctx.handle, pilot.handle, Yd.data_ptr(), F, M, N,
                                      w.K, w.L, dt, H.data_ptr(), C.c_void_p(stream))
        assert st == 0, f"call {call}: status {st}"
        assert pk.get_status(dev) == 0
        err = O.nmse(H.cpu().numpy(), H_ref.cpu().numpy())
        assert err <= TOL_Q[dtype], f"call {call}: NMSE {err:.3e} against pnce_estimate"
        # and the estimate itself is right
        assert O.nmse(H.cpu().numpy(), O.estimate_quantized(Y, bits, w.K, w.L, dtype)) <= TOL_Q[dtype]


def test_static_rejects_oversize_and_fp32(pk):
    dev = torch.device("cuda", 0)
    lib = pk.lib()
    N = 4095
    bits = np.zeros(N, dtype=np.uint8)
    bits[::3] = 1
    pilot = pk.Pilot(bits, device=dev)
    M, K, L = 128, 16, 128
    F = 1
    while pk.workspace_size(F, M, N, K, L, "fp16") <= STATIC_BYTES:
        F += 1
    Y = torch.zeros((F, M, N), dtype=torch.complex64, device=dev)
    H = torch.zeros((F, M, K, L), dtype=torch.complex64, device=dev)
    st = lib.pnce_estimate_static(pilot.ctx.handle, pilot.handle, Y.data_ptr(), F, M, N, K, L,
                                  pk.DTYPES["fp16"], H.data_ptr(), None)
    assert st == 1                                   # PNCE_EINVAL: does not fit
    st = lib.pnce_estimate_static(pilot.ctx.handle, pilot.handle, Y.data_ptr(), F - 1, M, N, K,
                                  L, pk.DTYPES["fp16"], H.data_ptr(), None)
    assert st == 0                                   # the largest batch that fits runs
    st = lib.pnce_estimate_static(pilot.ctx.handle, pilot.handle, Y.data_ptr(), 1, M, N, K, L,
                                  pk.DTYPES["fp32"], H.data_ptr(), None)
    assert st == 1                                   # FP32 SIMT has no scratch to place
    assert pk.get_status(dev) == 0
