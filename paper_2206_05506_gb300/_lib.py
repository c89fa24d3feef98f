"""ctypes binding of libpnce.so (the C ABI declared in include/pnce.h).

Argument marshalling only.  The library must have been built in-tree (build.py); if it
is missing, loading raises immediately: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB_PATH

PNCE_OK, PNCE_EINVAL, PNCE_EUNSUPPORTED, PNCE_ENOMEM, PNCE_ECUDA, PNCE_ETIMEOUT, PNCE_ESTATE = range(7)

DTYPES = {"fp32": 0, "tf32": 1, "fp16": 2, "bf16": 3, "e4m3": 4, "auto": 5}


class PnceError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = _lib.pnce_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{what}: {msg}")


_lib = None

_vp, _i, _sz = C.c_void_p, C.c_int, C.c_size_t


class ReqDesc(C.Structure):
    """pnce_req_desc: one request of a grouped estimate."""
    _fields_ = [("Y", C.c_void_p), ("H", C.c_void_p), ("M", C.c_int), ("K", C.c_int),
                ("L", C.c_int), ("row_offset", C.c_int)]


class FrameOpts(C.Structure):
    """pnce_frame_opts"""
    _fields_ = [("cp_len", C.c_int), ("shift_rule", C.c_int)]


class ServeReq(C.Structure):
    """pnce_serve_req: one request of a native serving run."""
    _fields_ = [("Y", C.c_void_p), ("H", C.c_void_p), ("M", C.c_int), ("N", C.c_int),
                ("K", C.c_int), ("L", C.c_int), ("t_arrival", C.c_double)]


class ServeOut(C.Structure):
    """pnce_serve_out: what a native serving run reports per request."""
    _fields_ = [("t_admit", C.c_double), ("t_launch", C.c_double), ("t_done", C.c_double),
                ("batch", C.c_int), ("status", C.c_int)]

_SIGS = {
    "pnce_version": (_i, []),
    "pnce_auto_dtype": (_i, [_i, _i, _i]),
    "pnce_status_string": (C.c_char_p, [_i]),
    "pnce_create": (_i, [C.POINTER(_vp)]),
    "pnce_destroy": (_i, [_vp]),
    "pnce_get_status": (_i, [_vp, _vp]),
    "pnce_pilot_create": (_i, [_vp, C.POINTER(C.c_uint32), _i, C.POINTER(_vp)]),
    "pnce_pilot_destroy": (_i, [_vp]),
    "pnce_workspace_size": (_sz, [_i, _i, _i, _i, _i, _i]),
    "pnce_estimate": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _vp, _sz, _vp, _vp]),
    "pnce_estimate_ex": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, C.POINTER(FrameOpts), _vp,
                              _sz, _vp, _vp]),
    "pnce_quantize": (_i, [_vp, _vp, _i, _i, _i, _i, _vp, _sz, _vp, _vp, _vp]),
    "pnce_correlate_quantized": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _i, _vp, _sz, _vp, _vp]),
    "pnce_estimate_real_pilot": (_i, [_vp, _vp, _i, _vp, _i, _i, _i, _i, _i, _vp, _vp]),
    "pnce_backward_workspace_size": (_sz, [_i, _i, _i, _i, _i]),
    "pnce_backward": (_i, [_vp, _vp, _i, _vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _vp, _sz, _vp]),
    "pnce_host_workspace_size": (_sz, [_i, _i, _i, _i, _i, _i]),
    "pnce_estimate_host": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _vp, _sz, _vp, _vp]),
    "pnce_estimate_static": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _vp, _vp]),
    "pnce_grouped_workspace_size": (_sz, [_i, _i, _i, _i]),
    "pnce_estimate_grouped": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _vp, _sz, _vp]),
    "pnce_fmt_tables": (_i, [C.POINTER(C.c_uint32), _i, C.POINTER(C.c_uint16),
                             C.POINTER(C.c_uint16)]),
    "pnce_fmt_create": (_i, [_vp, C.POINTER(C.c_uint32), _i, C.POINTER(_vp)]),
    "pnce_fmt_destroy": (_i, [_vp]),
    "pnce_estimate_fmt": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _vp, _vp]),
    "pnce_trace_enable": (_i, [_vp, _i]),
    "pnce_trace_read": (_i, [_vp, _vp, _vp, _i, C.POINTER(C.c_int)]),
    "pnce_gather_rows": (_i, [_vp, _i, _i, _vp, C.c_longlong, _vp]),
    "pnce_scatter_rows": (_i, [_vp, C.c_longlong, _vp, _vp, _i, _vp]),
    "pnce_server_create": (_i, [_vp, _i, _i, C.c_double, _i, C.POINTER(_vp)]),
    "pnce_server_destroy": (_i, [_vp]),
    "pnce_server_add_pilot": (_i, [_vp, _vp]),
    "pnce_server_prepare": (_i, [_vp, _i, _i, _i]),
    "pnce_server_run": (_i, [_vp, _vp, _i, _vp, C.POINTER(_i)]),
    "pnce_server_start": (_i, [_vp]),
    "pnce_server_submit": (_i, [_vp, C.POINTER(ServeReq), C.POINTER(C.c_longlong)]),
    "pnce_server_poll": (_i, [_vp, _vp, _vp, _i, C.POINTER(_i)]),
    "pnce_server_open": (_i, [_vp, C.POINTER(_i)]),
    "pnce_sched_simulate": (_i, [_vp, _i, _i, C.c_double, _i, C.c_double, C.c_double,
                                 C.c_double, C.c_double, _i, _i, _vp, C.POINTER(_i)]),
}


def exported_names() -> list[str]:
    return sorted(_SIGS)


def load(path: str | None = None):
    """Load libpnce.so (once) and declare every entry point's signature."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(
            f"libpnce.so not found at {path}: build it first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, what: str) -> None:
    if status != PNCE_OK:
        raise PnceError(status, what)
