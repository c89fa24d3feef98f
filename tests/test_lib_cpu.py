"""Host-side checks of the C ABI library that need no GPU: it builds, loads, exports
every function include/pnce.h declares, and its pure host functions behave."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pnce.h")


@pytest.fixture(scope="session")
def lib():
    from paper_2206_05506_gb300 import _lib, build

    if not os.path.exists(build.LIB_PATH):
        build.build()
    return _lib.load()


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pnce_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = header_functions()
    for must in ("pnce_estimate", "pnce_pilot_create", "pnce_quantize", "pnce_backward",
                 "pnce_correlate_quantized", "pnce_estimate_real_pilot", "pnce_estimate_host"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(lib):
    from paper_2206_05506_gb300 import _lib

    assert set(_lib.exported_names()) == set(header_functions())


def test_status_strings_and_version(lib):
    assert lib.pnce_version() >= 10000
    for s in range(7):
        assert lib.pnce_status_string(s).startswith(b"PNCE_")
    assert lib.pnce_status_string(99).startswith(b"PNCE_?")


def test_workspace_size_rules(lib):
    # FP32 SIMT needs no workspace; invalid shapes (Eq. 7: K*L > N) give 0
    assert lib.pnce_workspace_size(1, 8, 127, 2, 16, 0) == 0
    assert lib.pnce_workspace_size(1, 8, 127, 8, 16, 2) == 0
    assert lib.pnce_workspace_size(0, 8, 127, 2, 16, 2) == 0
    assert lib.pnce_workspace_size(1, 8, 127, 2, 16, 99) == 0
    # fp16: 16*ceil(F*M/8) rows (8-antenna groups) of ceil(N/64)*64 halfs, then F*M float
    # factors, 256-byte rounded
    F, M, N = 3, 5, 1023
    rows, pitch = 16 * ((F * M + 7) // 8), 1024
    a = rows * pitch * 2
    want = ((a + 255) // 256 * 256 + 4 * F * M + 255) // 256 * 256
    assert lib.pnce_workspace_size(F, M, N, 8, 64, 2) == want
    assert lib.pnce_workspace_size(F, M, N, 8, 64, 1) > lib.pnce_workspace_size(F, M, N, 8, 64, 2)
    assert lib.pnce_workspace_size(F, M, N, 8, 64, 4) < lib.pnce_workspace_size(F, M, N, 8, 64, 2)


def test_null_arguments_rejected_without_device(lib):
    # validation happens before any CUDA call
    assert lib.pnce_create(None) == 1
    assert lib.pnce_destroy(None) == 1
    assert lib.pnce_pilot_destroy(None) == 1
    assert lib.pnce_estimate(None, None, None, 1, 1, 7, 1, 1, 0, None, 0, None, None) == 1
    assert lib.pnce_backward(None, None, 0, None, None, 1, 1, 7, 1, 1, None, None, None, 0,
                             None) == 1


def test_serving_loop_rejects_bad_arguments_without_device(lib):
    # the native serving loop's entry points validate before any CUDA call
    import ctypes as C
    from paper_2206_05506_gb300 import _lib
    out = C.c_void_p()
    n = C.c_int(0)
    t = C.c_longlong(0)
    req = _lib.ServeReq(None, None, 4, 7, 1, 1, 0.0)
    assert lib.pnce_server_create(None, 2, 4, 1e9, 4096, C.byref(out)) == 1
    assert lib.pnce_server_destroy(None) == 1
    assert lib.pnce_server_add_pilot(None, None) == 1
    assert lib.pnce_server_prepare(None, 7, 4, 64) == 1
    assert lib.pnce_server_run(None, None, 0, None, C.byref(n)) == 1
    assert lib.pnce_server_start(None) == 1
    assert lib.pnce_server_submit(None, C.byref(req), C.byref(t)) == 1
    assert lib.pnce_server_poll(None, None, None, 0, C.byref(n)) == 1
    assert lib.pnce_server_open(None, C.byref(n)) == 1
    outs = (_lib.ServeOut * 1)()
    bad = (_lib.ServeReq * 1)(_lib.ServeReq(None, None, 4, 7, 8, 1, 0.0))   # K*L > N
    assert lib.pnce_sched_simulate(bad, 1, 2, 1e9, 4096, 1000.0, 2e-4, 2e-7, 5e-6, 0, 0,
                                   outs, C.byref(n)) == 1
    ok = (_lib.ServeReq * 1)(_lib.ServeReq(None, None, 4, 7, 1, 1, 0.0))
    assert lib.pnce_sched_simulate(ok, 1, 0, 1e9, 4096, 1000.0, 2e-4, 2e-7, 5e-6, 0, 0,
                                   outs, C.byref(n)) == 1                 # no slot
    assert lib.pnce_sched_simulate(ok, 1, 2, 1e9, 4096, 1000.0, 2e-4, 2e-7, 5e-6, -1, 0,
                                   outs, C.byref(n)) == 1                 # bad fault period
    assert lib.pnce_sched_simulate(ok, 1, 2, 1e9, 4096, 1000.0, 2e-4, 2e-7, 5e-6, 0, 0,
                                   outs, C.byref(n)) == 0 and n.value == 1
    assert outs[0].status == 0 and outs[0].t_done > outs[0].t_launch >= 0.0


def test_missing_library_fails_loudly():
    # no CPU or PyTorch fallback: without the built library the binding refuses to run
    from paper_2206_05506_gb300 import _lib
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="libpnce.so not found"):
            _lib.load(os.path.join(ROOT, "no_such_directory", "libpnce.so"))
    finally:
        _lib._lib = saved


def test_new_entry_points_validate_before_any_device_use(lib):
    # grouped serving estimate and the transform yardstick reject bad arguments up front
    assert lib.pnce_estimate_grouped(None, None, None, 1, 64, 32, 2, None, 0, None) == 1
    assert lib.pnce_grouped_workspace_size(0, 127, 16, 2) == 0          # no rows
    assert lib.pnce_grouped_workspace_size(64, 127, 128, 2) == 0        # kl_max > N
    assert lib.pnce_grouped_workspace_size(64, 127, 16, 99) == 0        # unknown dtype
    assert lib.pnce_grouped_workspace_size(64, 127, 16, 0) > 0
    assert lib.pnce_fmt_create(None, None, 127, None) == 1
    assert lib.pnce_fmt_destroy(None) == 1
    assert lib.pnce_estimate_fmt(None, None, None, 1, 1, 127, 1, 1, None, None) == 1
    assert lib.pnce_estimate_static(None, None, None, 1, 1, 127, 1, 1, 2, None, None) == 1


def test_product_code_does_not_import_the_oracle():
    # the oracle is test infrastructure: nothing under the package may import it
    pkg = os.path.join(ROOT, "paper_2206_05506_gb300")
    pat = re.compile(r"^\s*(import|from)\s+oracle\b", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                assert not pat.search(open(os.path.join(dirpath, f)).read()), f


def test_empty_and_degenerate_shapes_rejected_up_front(lib):
    # F = 0 or M = 0 (empty batch), N < 2, K or L = 0, and K*L > N (Eq. 7) are PNCE_EINVAL
    # and need no workspace; the shape is checked before any pointer is used, so stand-in
    # addresses are never dereferenced
    dummy = C.c_void_p(256)
    for F, M, N, K, L in [(0, 4, 127, 1, 8), (1, 0, 127, 1, 8), (1, 4, 1, 1, 1),
                          (1, 4, 127, 0, 8), (1, 4, 127, 1, 0), (1, 4, 127, 2, 64)]:
        for dt in (1, 2, 3, 4):
            assert lib.pnce_workspace_size(F, M, N, K, L, dt) == 0
        assert lib.pnce_backward_workspace_size(F, M, N, K, L) == 0
        for dt in (0, 2):
            assert lib.pnce_estimate(dummy, dummy, dummy, F, M, N, K, L, dt, dummy, 1 << 30,
                                     dummy, None) == 1
    # the full-lag case K*L = N is admissible
    assert lib.pnce_workspace_size(1, 4, 127, 1, 127, 2) > 0


def test_binding_refuses_bad_output_buffers_before_launch():
    # output and workspace pointers go to the kernels unchecked, so the Python wrappers
    # must refuse a buffer of the wrong shape, dtype, device or layout up front
    import torch
    import paper_2206_05506_gb300 as pk

    cpu = torch.device("cpu")
    shape = (2, 3, 4, 5)
    good = torch.empty(shape, dtype=torch.complex64)
    assert pk._check_out(good, shape, cpu) is good
    bad = [torch.empty((2, 3, 4, 4), dtype=torch.complex64),           # too small
           torch.empty((2, 3, 4, 6), dtype=torch.complex64),           # wrong shape
           torch.empty(shape, dtype=torch.complex128),                 # wrong dtype
           torch.empty(shape, dtype=torch.float32),
           torch.empty((2, 3, 5, 4), dtype=torch.complex64).transpose(2, 3),  # strided
           torch.empty(shape, dtype=torch.complex64, device="meta"),   # another device
           "not a tensor"]
    for b in bad:
        with pytest.raises(ValueError):
            pk._check_out(b, shape, cpu)
    with pytest.raises(ValueError):                 # a host buffer where a GPU one is due
        pk._check_out(good, shape, torch.device("cuda", 0))
    with pytest.raises(ValueError):                 # a pilot of the wrong length
        pk._check_out(torch.empty(7), (8,), cpu, what="p", dtype=torch.float32)
    ws = torch.empty(100, dtype=torch.uint8)
    assert pk._check_workspace(ws, cpu, 100) is ws
    assert pk._check_workspace(torch.empty(25, dtype=torch.float32), cpu, 100) is not None
    for b, need in [(ws, 101), (torch.empty(100, dtype=torch.uint8, device="meta"), 10),
                    (torch.empty(200, dtype=torch.uint8)[::2], 10)]:
        with pytest.raises(ValueError):
            pk._check_workspace(b, cpu, need)


def test_auto_dtype_rule(lib):
    # PNCE_AUTO: exact FP32 on the CUDA cores up to 16 lags, fp16 tensor cores above
    assert lib.pnce_auto_dtype(127, 1, 1) == 0
    assert lib.pnce_auto_dtype(127, 2, 8) == 0
    assert lib.pnce_auto_dtype(127, 1, 17) == 2
    assert lib.pnce_auto_dtype(4095, 16, 128) == 2
    assert lib.pnce_auto_dtype(127, 2, 64) == -1            # K*L > N: invalid shape
    assert lib.pnce_auto_dtype(1, 1, 1) == -1
    for F, M, N, K, L in [(3, 5, 1023, 2, 8), (3, 5, 1023, 8, 64), (1, 130, 4095, 16, 128)]:
        want = lib.pnce_auto_dtype(N, K, L)
        assert lib.pnce_workspace_size(F, M, N, K, L, 5) == lib.pnce_workspace_size(F, M, N, K, L, want)
        assert lib.pnce_host_workspace_size(F, M, N, K, L, 5) == \
            lib.pnce_host_workspace_size(F, M, N, K, L, want)
    assert lib.pnce_grouped_workspace_size(64, 1023, 16, 5) == lib.pnce_grouped_workspace_size(64, 1023, 16, 0)
    assert lib.pnce_grouped_workspace_size(64, 1023, 64, 5) == lib.pnce_grouped_workspace_size(64, 1023, 64, 2)
    # the entry points that name one tensor-core step or format do not take it
    dummy = C.c_void_p(256)
    assert lib.pnce_quantize(dummy, dummy, 1, 8, 127, 5, dummy, 1 << 20, None, None, None) == 1
    assert lib.pnce_estimate_static(dummy, dummy, dummy, 1, 8, 127, 2, 16, 5, dummy, None) == 1
