"""Oracle side of the full-size parity test (not collected by pytest: no test_ prefix).

One call handles one chunk of frames of the precision workload: it regenerates the
chunk's received blocks from the workload seed (the generator is per frame, so the
chunk is the same data the GPU saw), computes the FP64 oracle and the oracle on each
quantised operand, and compares them with the GPU estimates of the chunk that the
parent process passes in.  It returns per-frame sums, so the parent can form NMSE per
frame, per SNR and per launch.

Runs in worker processes started with the 'spawn' method: they import numpy, the oracle
and the generator only, never torch or the CUDA library.
"""
from __future__ import annotations

import numpy as np

from oracle import pn_oracle as O
from synth import channel as C


def chunk_stats(first: int, frames: int, gpu: dict) -> dict:
    """{dtype: (num_plain, num_q, den_plain, den_q)} per frame of [first, first+frames).

    num_plain = sum |H_gpu - H_oracle|^2, den_plain = sum |H_oracle|^2 (per frame);
    num_q / den_q the same against the oracle on the dtype's quantised operand.
    """
    w = C.PRECISION
    bits, Y = C.make_received(w, frames=frames, first=first)
    ref = O.estimate(Y, bits, w.K, w.L)
    den = (np.abs(ref) ** 2).sum(axis=(1, 2, 3))
    out = {}
    for dtype, Hc in gpu.items():
        H = np.asarray(Hc).astype(np.complex128)
        num = (np.abs(H - ref) ** 2).sum(axis=(1, 2, 3))
        if dtype == "fp32":
            numq, denq = num, den
            out["fp32_maxabs"] = float(np.abs(H - ref).max() / np.abs(ref).max())
        else:
            refq = O.estimate_quantized(Y, bits, w.K, w.L, dtype)
            numq = (np.abs(H - refq) ** 2).sum(axis=(1, 2, 3))
            denq = (np.abs(refq) ** 2).sum(axis=(1, 2, 3))
        out[dtype] = (num, numq, den, denq)
    return out
