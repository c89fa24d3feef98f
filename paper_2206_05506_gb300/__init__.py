"""PN-sequence correlation channel estimation on GB300 (sm_103a).

Python face of libpnce (include/pnce.h).  PyTorch supplies device memory and streams;
every step of the estimator runs in the library's CUDA kernels:

    H[f, m, k, l] = (1/N) sum_n Y[f, m, n] p[(n - l - k L) mod N]

(the correlator (1/N) S^T Y of Eq. 3 / Eq. 10 with K transmitters multiplexed by the
cyclic shifts k*L of one m-sequence, Sec. II-B).

    pilot = Pilot(bits)                       # 0/1 m-sequence bits, uploaded once
    H = estimate(Y, pilot, K, L, dtype="fp16")  # Y: complex64 CUDA tensor [F, M, N]

dtype: "fp32" (exact FP32 on the CUDA cores), or "tf32" / "fp16" / "bf16" / "e4m3"
(per-antenna power-of-two scaled operand, tensor cores, FP32 accumulation).
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np
import torch

from . import _lib
from ._lib import DTYPES, PnceError, check

__all__ = ["Pilot", "Context", "estimate", "quantize", "correlate_quantized",
           "estimate_real_pilot", "backward", "estimate_host", "PILOT_MAPS", "workspace_size",
           "host_workspace_size", "backward_workspace_size", "get_status", "DTYPES",
           "trace_enable", "trace_read",
           "PnceError", "lib"]


def lib():
    return _lib.load()


def _dt(dtype) -> int:
    if isinstance(dtype, int):
        return dtype
    try:
        return DTYPES[dtype]
    except KeyError:
        raise ValueError(f"unknown dtype {dtype!r}; one of {sorted(DTYPES)}") from None


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


class Context:
    """A pnce_handle bound to one CUDA device (latched device status word)."""

    def __init__(self, device=None):
        d = None if device is None else torch.device("cuda", device) if isinstance(device, int) \
            else torch.device(device)
        idx = d.index if d is not None and d.index is not None else torch.cuda.current_device()
        self.device = torch.device("cuda", idx)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            check(lib().pnce_create(C.byref(h)), "pnce_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def status(self, stream=None) -> int:
        with torch.cuda.device(self.device):
            s = _stream(self.device) if stream is None else stream
            return lib().pnce_get_status(self._h, s)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib._lib is not None:
            _lib._lib.pnce_destroy(h)
            self._h = None


_ctx_lock = threading.Lock()
_contexts: dict[int, Context] = {}


def context(device=None) -> Context:
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    idx = dev.index if dev.index is not None else torch.cuda.current_device()
    with _ctx_lock:
        if idx not in _contexts:
            _contexts[idx] = Context(idx)
        return _contexts[idx]


def trace_enable(on: bool = True, device=None):
    """Record CUDA events around every kernel the estimate entry points launch."""
    ctx = context(device)
    check(lib().pnce_trace_enable(ctx.handle, 1 if on else 0), "pnce_trace_enable")


TRACE_KINDS = {0: "quantize", 1: "correlate", 2: "simt", 3: "fmt", 4: "adjoint"}


def trace_read(device=None, max_entries: int = 8192):
    """[(kind, ms)] of the kernels traced since the last read (waits for them)."""
    ctx = context(device)
    kinds = (C.c_int * max_entries)()
    ms = (C.c_float * max_entries)()
    n = C.c_int(0)
    check(lib().pnce_trace_read(ctx.handle, kinds, ms, max_entries, C.byref(n)),
          "pnce_trace_read")
    return [(TRACE_KINDS.get(kinds[i], str(kinds[i])), float(ms[i])) for i in range(n.value)]


def get_status(device=None) -> int:
    """Synchronise the current stream and return (and clear) the latched device status."""
    return context(device).status()


class Pilot:
    """Device-resident m-sequence pilot (bits 0/1, bit 0 -> +1, bit 1 -> -1)."""

    def __init__(self, bits, device=None):
        self.N, self.words = _pack_bits(bits)
        self.ctx = context(device)
        self.device = self.ctx.device
        p = C.c_void_p()
        with torch.cuda.device(self.device):
            check(lib().pnce_pilot_create(self.ctx.handle,
                                          self.words.ctypes.data_as(C.POINTER(C.c_uint32)),
                                          self.N, C.byref(p)), "pnce_pilot_create")
        self._p = p

    @property
    def handle(self):
        return self._p

    def __del__(self):
        p = getattr(self, "_p", None)
        if p is not None and _lib._lib is not None:
            _lib._lib.pnce_pilot_destroy(p)
            self._p = None


def _pack_bits(bits) -> tuple[int, np.ndarray]:
    b = np.asarray(bits.cpu().numpy() if isinstance(bits, torch.Tensor) else bits)
    b = b.astype(np.uint8).ravel()
    if b.size < 2 or np.any(b > 1):
        raise ValueError("pilot bits must be a 0/1 array of length >= 2")
    nw = (b.size + 31) // 32
    padded = np.zeros(nw * 32, dtype=np.uint64)
    padded[: b.size] = b
    words = (padded.reshape(nw, 32) << np.arange(32, dtype=np.uint64)).sum(axis=1)
    return int(b.size), np.ascontiguousarray(words.astype(np.uint32))


def fmt_tables(bits):
    """(pos, lagvec) uint16 arrays of the fast m-sequence transform (host only): the r-bit
    window s_n of every sample n and the vector u_j of every lag j, with
    bit[(n - j) mod N] = parity(u_j & s_n).  Raises PnceError unless bits is an m-sequence."""
    N, words = _pack_bits(bits)
    pos = np.zeros(N, dtype=np.uint16)
    lag = np.zeros(N, dtype=np.uint16)
    check(lib().pnce_fmt_tables(words.ctypes.data_as(C.POINTER(C.c_uint32)), N,
                                pos.ctypes.data_as(C.POINTER(C.c_uint16)),
                                lag.ctypes.data_as(C.POINTER(C.c_uint16))), "pnce_fmt_tables")
    return pos, lag


class FmtPilot:
    """Device tables of the fast m-sequence transform (a yardstick, not the paper's method)."""

    def __init__(self, bits, device=None):
        self.N, words = _pack_bits(bits)
        self.ctx = context(device)
        self.device = self.ctx.device
        p = C.c_void_p()
        with torch.cuda.device(self.device):
            check(lib().pnce_fmt_create(self.ctx.handle,
                                        words.ctypes.data_as(C.POINTER(C.c_uint32)), self.N,
                                        C.byref(p)), "pnce_fmt_create")
        self._p = p

    @property
    def handle(self):
        return self._p

    def __del__(self):
        p = getattr(self, "_p", None)
        if p is not None and _lib._lib is not None:
            _lib._lib.pnce_fmt_destroy(p)
            self._p = None


def estimate_fmt(Y: torch.Tensor, fmt: "FmtPilot", K: int, L: int, out=None) -> torch.Tensor:
    """The estimate by the fast m-sequence transform (FP32, CUDA cores): same H as
    estimate(), computed in O(N log N) per row."""
    F, M, N = _check_y(Y)
    if N != fmt.N:
        raise ValueError("Y's N differs from the transform's")
    dev = Y.device
    H = _out_or_new(out, (F, M, K, L), dev)
    with torch.cuda.device(dev):
        check(lib().pnce_estimate_fmt(fmt.ctx.handle, fmt.handle, Y.data_ptr(), F, M, N, K, L,
                                      H.data_ptr(), _stream(dev)), "pnce_estimate_fmt")
    return H


def workspace_size(F, M, N, K, L, dtype) -> int:
    return int(lib().pnce_workspace_size(F, M, N, K, L, _dt(dtype)))


def grouped_workspace_size(rows, N, kl_max, dtype) -> int:
    return int(lib().pnce_grouped_workspace_size(rows, N, kl_max, _dt(dtype)))


def estimate_grouped(pilot: "Pilot", descs_ptr: int, nreq: int, rows: int, kl_max: int, dtype,
                     workspace: torch.Tensor, stream=None):
    """Grouped estimate (pnce_estimate_grouped): descs_ptr is the address of nreq
    pnce_req_desc entries (_lib.ReqDesc) that the GPU can read (device or page-locked
    host memory); each request's Y and H buffers likewise.  Enqueues only."""
    dev = pilot.device
    _check_workspace(workspace, dev, grouped_workspace_size(rows, pilot.N, kl_max, dtype))
    with torch.cuda.device(dev):
        s = _stream(dev) if stream is None else stream
        check(lib().pnce_estimate_grouped(pilot.ctx.handle, pilot.handle, descs_ptr, nreq, rows,
                                          kl_max, _dt(dtype), workspace.data_ptr(),
                                          workspace.numel() * workspace.element_size(), s),
              "pnce_estimate_grouped")


def backward_workspace_size(F, M, N, K, L) -> int:
    return int(lib().pnce_backward_workspace_size(F, M, N, K, L))


def host_workspace_size(F, M, N, K, L, dtype) -> int:
    return int(lib().pnce_host_workspace_size(F, M, N, K, L, _dt(dtype)))


_ws_cache: dict[tuple, torch.Tensor] = {}


def _workspace(device, nbytes: int, key=None) -> torch.Tensor | None:
    """A cached byte buffer per (device, stream, key), grown on demand."""
    if nbytes == 0:
        return None
    k = (device.index, _stream(device), key)
    buf = _ws_cache.get(k)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        _ws_cache[k] = buf
    return buf


def _check_y(Y: torch.Tensor, pilot: Pilot | None = None):
    if not isinstance(Y, torch.Tensor) or Y.dtype != torch.complex64 or Y.dim() != 3:
        raise ValueError("Y must be a complex64 tensor [F, M, N]")
    if not Y.is_cuda:
        raise ValueError("Y must be a CUDA tensor (use estimate_host for host buffers)")
    if not Y.is_contiguous():
        raise ValueError("Y must be contiguous")
    if pilot is not None and Y.shape[2] != pilot.N:
        raise ValueError(f"Y has N={Y.shape[2]} samples but the pilot has N={pilot.N}")
    return Y.shape


def _check_out(out, shape, device, what="out", dtype=torch.complex64):
    """`out` if it is a contiguous `dtype` tensor of `shape` on `device`, else ValueError.

    Output and workspace pointers go to the kernels unchecked, so a buffer that is too
    small, strided, or on another device must be refused here, before any launch."""
    if not isinstance(out, torch.Tensor):
        raise ValueError(f"{what} must be a torch.Tensor")
    if out.dtype != dtype or tuple(out.shape) != tuple(shape):
        raise ValueError(f"{what} must be a {dtype} tensor of shape {tuple(shape)}, "
                         f"got {out.dtype} {tuple(out.shape)}")
    if out.device != device:
        raise ValueError(f"{what} is on {out.device}, expected {device}")
    if not out.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return out


def _out_or_new(out, shape, device, pin_memory=False):
    if out is None:
        if device.type == "cpu":
            return torch.empty(shape, dtype=torch.complex64, pin_memory=pin_memory)
        return torch.empty(shape, dtype=torch.complex64, device=device)
    return _check_out(out, shape, device)


def _check_workspace(ws, device, need, what="workspace"):
    """A caller-supplied workspace: a contiguous tensor on `device` of >= need bytes."""
    if ws is None:
        return None
    if not isinstance(ws, torch.Tensor) or ws.device != device or not ws.is_contiguous():
        raise ValueError(f"{what} must be a contiguous tensor on {device}")
    if ws.numel() * ws.element_size() < need:
        raise ValueError(f"{what} holds {ws.numel() * ws.element_size()} bytes, "
                         f"{need} needed")
    return ws


SHIFT_RULES = {"kl": 0, "spread": 1}


def estimate(Y: torch.Tensor, pilot: Pilot, K: int, L: int, dtype="fp32", out=None,
             workspace: torch.Tensor | None = None, cp_len: int = 0,
             shift_rule: str = "kl") -> torch.Tensor:
    """Channel estimate H [F, M, K, L] (complex64) of received blocks Y [F, M, cp_len + N].

    cp_len: cyclic-prefix samples at the head of each row (skipped).  shift_rule: "kl"
    (transmitter k at cyclic shift k*L) or "spread" (k*floor(N/K), Eq. 8).
    """
    if cp_len == 0 and shift_rule == "kl":
        F, M, N = _check_y(Y, pilot)
    else:
        F, M, T = _check_y(Y)
        N = pilot.N
        if T != cp_len + N:
            raise ValueError(f"rows hold {T} samples, expected cp_len + N = {cp_len + N}")
    dt = _dt(dtype)
    dev = Y.device
    H = _out_or_new(out, (F, M, K, L), dev)
    need = workspace_size(F, M, N, K, L, dt)
    ws = _check_workspace(workspace, dev, need) if workspace is not None \
        else _workspace(dev, need)
    nbytes = 0 if ws is None else ws.numel() * ws.element_size()
    with torch.cuda.device(dev):
        if cp_len == 0 and shift_rule == "kl":
            check(lib().pnce_estimate(pilot.ctx.handle, pilot.handle, Y.data_ptr(), F, M, N, K,
                                      L, dt, _ptr(ws), nbytes, H.data_ptr(), _stream(dev)),
                  "pnce_estimate")
        else:
            opts = _lib.FrameOpts(cp_len, SHIFT_RULES[shift_rule])
            check(lib().pnce_estimate_ex(pilot.ctx.handle, pilot.handle, Y.data_ptr(), F, M, N,
                                         K, L, dt, C.byref(opts), _ptr(ws), nbytes, H.data_ptr(),
                                         _stream(dev)), "pnce_estimate_ex")
    return H


def operand_rows(A: int):
    """Row indices (real, imaginary) of antennas 0..A-1 in the quantised operand."""
    a = torch.arange(A, dtype=torch.int64)
    re = 16 * (a // 8) + a % 8
    return re, re + 8


def quantize(Y: torch.Tensor, dtype, workspace=None, want_power=False):
    """Run only the quantisation step; returns a dict of views into the workspace.

    'q': the operand as raw integer codes [16*ceil(F*M/8), pitch] (uint16 for fp16/bf16,
    int32 for tf32, uint8 for e4m3) in groups of 8 antennas: row 16*(a//8) + a%8 holds the
    real part of antenna a = f*M + m, row 16*(a//8) + 8 + a%8 its imaginary part
    (operand_rows() gives the row indices); 'factor': float32 [F*M] = 2^-s / N, 'exps':
    int32 s, 'power': float64 mean power (if want_power), 'workspace': the buffer.
    """
    F, M, N = _check_y(Y)
    dt = _dt(dtype)
    if dt == 0:
        raise ValueError("fp32 has no quantised operand")
    dev = Y.device
    need = workspace_size(F, M, N, 1, 1, dt)
    ws = _check_workspace(workspace, dev, need) if workspace is not None \
        else torch.empty(need, dtype=torch.uint8, device=dev)
    exps = torch.empty(F * M, dtype=torch.int32, device=dev)
    power = torch.empty(F * M, dtype=torch.float64, device=dev) if want_power else None
    with torch.cuda.device(dev):
        check(lib().pnce_quantize(context(dev).handle, Y.data_ptr(), F, M, N, dt, ws.data_ptr(),
                                  ws.numel() * ws.element_size(), exps.data_ptr(), _ptr(power),
                                  _stream(dev)),
              "pnce_quantize")
    pitch = (N + 63) // 64 * 64
    eb = {1: 4, 2: 2, 3: 2, 4: 1}[dt]
    rows = 16 * ((F * M + 7) // 8)
    abytes = rows * pitch * eb
    view_dt = {4: torch.int32, 2: torch.int16, 1: torch.uint8}[eb]
    q = ws[:abytes].view(view_dt).view(rows, pitch)
    sc_off = (abytes + 255) // 256 * 256
    factor = ws[sc_off:sc_off + 4 * F * M].view(torch.float32)
    return {"q": q, "factor": factor, "exps": exps, "power": power, "workspace": ws,
            "pitch": pitch}


def correlate_quantized(workspace: torch.Tensor, pilot: Pilot, F, M, K, L, dtype, out=None):
    """Tensor-core correlation of an operand already produced by quantize()."""
    dt = _dt(dtype)
    dev = pilot.device
    N = pilot.N
    _check_workspace(workspace, dev, workspace_size(F, M, N, K, L, dt))
    H = _out_or_new(out, (F, M, K, L), dev)
    with torch.cuda.device(dev):
        check(lib().pnce_correlate_quantized(pilot.ctx.handle, pilot.handle, F, M, N, K, L, dt,
                                             workspace.data_ptr(),
                                             workspace.numel() * workspace.element_size(),
                                             H.data_ptr(), _stream(dev)),
              "pnce_correlate_quantized")
    return H


PILOT_MAPS = {"real": 0, "tanh": 1}


def estimate_real_pilot(Y: torch.Tensor, p: torch.Tensor, K: int, L: int, out=None,
                        pilot_map: str = "real"):
    """FP32 estimate with a real-valued pilot (float32 CUDA tensor [N]).

    pilot_map="tanh": p holds theta and the pilot is tanh(theta), formed in the kernel.
    """
    F, M, N = _check_y(Y)
    if p.dtype != torch.float32 or p.shape != (N,) or not p.is_contiguous() or p.device != Y.device:
        raise ValueError("p must be a contiguous float32 tensor [N] on Y's device")
    dev = Y.device
    H = _out_or_new(out, (F, M, K, L), dev)
    with torch.cuda.device(dev):
        check(lib().pnce_estimate_real_pilot(context(dev).handle, p.data_ptr(),
                                             PILOT_MAPS[pilot_map], Y.data_ptr(), F, M, N, K, L,
                                             H.data_ptr(), _stream(dev)),
              "pnce_estimate_real_pilot")
    return H


def backward(p: torch.Tensor, Y: torch.Tensor, G: torch.Tensor, K: int, L: int,
             need_dY=True, need_dp=True, pilot_map: str = "real"):
    """Adjoint of estimate_real_pilot: (dY [F, M, N] complex64, dpilot [N] float32).

    With pilot_map="tanh" the second output is the gradient with respect to theta.
    """
    F, M, N = _check_y(Y)
    dev = Y.device
    _check_out(G, (F, M, K, L), dev, what="G")
    _check_out(p, (N,), dev, what="p", dtype=torch.float32)
    dY = torch.empty((F, M, N), dtype=torch.complex64, device=dev) if need_dY else None
    dp = torch.empty(N, dtype=torch.float32, device=dev) if need_dp else None
    need = backward_workspace_size(F, M, N, K, L) if need_dp else 0
    ws = _workspace(dev, need, key="bwd")
    with torch.cuda.device(dev):
        check(lib().pnce_backward(context(dev).handle, p.data_ptr(), PILOT_MAPS[pilot_map],
                                  Y.data_ptr(), G.data_ptr(), F, M, N, K, L, _ptr(dY), _ptr(dp),
                                  _ptr(ws), 0 if ws is None else ws.numel() * ws.element_size(),
                                  _stream(dev)),
              "pnce_backward")
    return dY, dp


def estimate_host(Y_host: torch.Tensor, pilot: Pilot, K: int, L: int, dtype="fp32", out=None,
                  workspace=None) -> torch.Tensor:
    """End-to-end estimate from a host complex64 tensor (pinned memory recommended).

    The C entry point copies Y to the device, estimates and copies H back, all on the
    current stream; this call waits for the result.
    """
    if Y_host.is_cuda or Y_host.dtype != torch.complex64 or Y_host.dim() != 3:
        raise ValueError("Y_host must be a host complex64 tensor [F, M, N]")
    Y_host = Y_host.contiguous()
    F, M, N = Y_host.shape
    dt = _dt(dtype)
    dev = pilot.device
    if N != pilot.N:
        raise ValueError(f"Y_host has N={N} samples but the pilot has N={pilot.N}")
    H = _out_or_new(out, (F, M, K, L), torch.device("cpu"), pin_memory=Y_host.is_pinned())
    need = host_workspace_size(F, M, N, K, L, dt)
    ws = _check_workspace(workspace, dev, need) if workspace is not None \
        else _workspace(dev, need, key="host")
    with torch.cuda.device(dev):
        s = _stream(dev)
        check(lib().pnce_estimate_host(pilot.ctx.handle, pilot.handle, Y_host.data_ptr(), F, M,
                                       N, K, L, dt, _ptr(ws),
                                       0 if ws is None else ws.numel() * ws.element_size(),
                                       H.data_ptr(), s), "pnce_estimate_host")
        torch.cuda.current_stream(dev).synchronize()
    return H
