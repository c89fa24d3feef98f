"""Synthetic reproduction of the paper's experiments (Sec. IV, Table I) on GB300.

The paper's figures carry no printed numbers, so these runs report what the same
experiments give here, with the paper's setup: N_t = N_r antennas, multiplexed pilot
slots of N_batch transmitters (cyclic shifts k*L of one m-sequence), CP length C = L,
channels of L_nz equal-variance taps at uniform positions inside L (Sec. II), 50
iterations per point (Table I).

  fig4  MAE (Eq. 12) vs SNR, PN length 511 / 2047, N_batch 1 / 2 / 4, L = L_nz = 64, 16x16
  fig5  MAE vs SNR, PN 2047, N_batch 4, L = 128, L_nz in {1, 16, 64, 128}, 16x16
  fig6  frame latency (host -> device copy + estimate + copy back) vs N_batch, PN
        511 / 1023 / 2047, L = 64, 16x16, against the frame propagation time of Eq. 11 at
        a 10 MHz sampling rate
  fig7  the same for 32x32 and 64x64, PN 2047, L = 128, L_nz = 20

A frame holds all N_t / N_batch pilot slots of the N_t transmitters (Sec. IV-C): one
estimate call of F = N_t / N_batch slots, M = N_r, K = N_batch.

    python paper_experiments.py [--dtype fp16] [--iters 50] [--out results.json]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import channel as C  # noqa: E402
from synth import mseq  # noqa: E402


def frame_inputs(rng, r, Nr, Nt, nb, L, lnz, snr_db):
    """One frame: Nt/nb slots; slot s carries transmitters s*nb .. s*nb+nb-1."""
    N = (1 << r) - 1
    bits = mseq.mseq_bits(r, 0)
    slots = Nt // nb
    h = C.channel(rng, slots, Nr, nb, L, lnz=lnz)          # [slots, Nr, nb, L]
    y = C.received(h, bits, snr_db, rng)                    # [slots, Nr, N]
    return bits, h, y, N


def mae_curve(pk, dev, r, Nr, Nt, nb, L, lnz, snrs, iters, dtype, seed=0):
    import torch
    out = []
    pilot = None
    for snr in snrs:
        errs = []
        for it in range(iters):
            rng = np.random.default_rng([seed, r, nb, L, lnz, int(snr * 10) + 1000, it])
            bits, h, y, N = frame_inputs(rng, r, Nr, Nt, nb, L, lnz, snr)
            if pilot is None:
                pilot = pk.Pilot(bits, device=dev)
            H = pk.estimate(torch.from_numpy(y).to(dev), pilot, nb, L, dtype=dtype)
            errs.append(np.mean(np.abs(H.cpu().numpy() - h)))     # Eq. 12
        out.append(float(np.mean(errs)))
    return out


def latency_curve(pk, dev, r, Nr, Nt, L, lnz, dtype, iters, fs_hz=10e6):
    """Per N_batch: median frame latency through pnce_estimate_host (copy in, estimate,
    copy out) and the frame propagation time P * N_t / (N_batch F_s) of Eq. 11."""
    import torch
    N = (1 << r) - 1
    rows = []
    for nb in (1, 2, 4, 8):
        if nb * L > N or Nt % nb:
            continue
        rng = np.random.default_rng([1, r, nb, Nr])
        bits, h, y, _ = frame_inputs(rng, r, Nr, Nt, nb, L, lnz, 20.0)
        pilot = pk.Pilot(bits, device=dev)
        Yh = torch.from_numpy(y).pin_memory()
        Hh = torch.empty((Nt // nb, Nr, nb, L), dtype=torch.complex64, pin_memory=True)
        ws = torch.empty(pk.host_workspace_size(Nt // nb, Nr, N, nb, L, dtype), dtype=torch.uint8,
                         device=dev)
        ts = []
        for it in range(iters + 5):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pk.estimate_host(Yh, pilot, nb, L, dtype=dtype, out=Hh, workspace=ws)
            ts.append(time.perf_counter() - t0)
        lat = float(np.median(ts[5:]))
        P = N + L                                       # pilot with CP, C = L (Sec. II-B)
        t_pr = P / fs_hz * Nt / nb                      # Eq. 11
        rows.append({"N_batch": nb, "latency_ms": lat * 1e3, "t_pr_ms_10MHz": t_pr * 1e3,
                     "frame_bytes_in": int(y.nbytes), "realtime_at_10MHz": lat <= t_pr})
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dtype", default="fp16")
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()

    import torch

    import paper_2206_05506_gb300 as pk
    dev = torch.device("cuda", 0)
    snrs = [-10.0, 0.0, 10.0, 20.0, 30.0, 40.0]
    res = {"dtype": args.dtype, "iters": args.iters, "snr_db": snrs}
    res["fig4"] = {f"pn{(1 << r) - 1}_nb{nb}": mae_curve(pk, dev, r, 16, 16, nb, 64, 64, snrs,
                                                          args.iters, args.dtype)
                   for r in (9, 11) for nb in (1, 2, 4)}
    res["fig5"] = {f"lnz{lnz}": mae_curve(pk, dev, 11, 16, 16, 4, 128, lnz, snrs, args.iters,
                                           args.dtype)
                   for lnz in (1, 16, 64, 128)}
    res["fig5_fp32"] = {f"lnz{lnz}": mae_curve(pk, dev, 11, 16, 16, 4, 128, lnz, snrs,
                                                args.iters, "fp32")
                        for lnz in (1, 128)}
    res["fig6"] = {f"pn{(1 << r) - 1}": latency_curve(pk, dev, r, 16, 16, 64, 64, args.dtype,
                                                       args.iters)
                   for r in (9, 10, 11)}
    res["fig7"] = {f"mimo{n}x{n}": latency_curve(pk, dev, 11, n, n, 128, 20, args.dtype,
                                                  args.iters)
                   for n in (32, 64)}
    txt = json.dumps(res, indent=1)
    print(txt)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(txt)


if __name__ == "__main__":
    main()
