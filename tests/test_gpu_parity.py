"""GPU parity of every estimator path against the FP64 oracle, through the C ABI.

Tolerances (NMSE = sum|gpu - ref|^2 / sum|ref|^2 over the launch):
* against the oracle on the unquantised complex64 input (the stated accuracy targets):
  1e-6 for the FP32 paths (SIMT, TF32), 2e-3 for FP16/BF16, 3e-2 for FP8-e4m3;
* against the oracle applied to the quantised operand (isolates the FP32 accumulation of
  the tensor-core product from the input rounding): 1e-9 for fp16/bf16/tf32 and 1e-6
  for e4m3 (whose accumulation inside the tensor core may keep fewer bits);
* the quantiser itself is integer/byte work and must match bit for bit.
Output buffers carry guard words on both sides, checked after every launch.
"""
import numpy as np
import pytest
import torch

from oracle import pn_oracle as O
from synth import channel as C

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-6, "tf32": 1e-6, "fp16": 2e-3, "bf16": 2e-3, "e4m3": 3e-2}
TOL_Q = {"tf32": 1e-9, "fp16": 1e-9, "bf16": 1e-9, "e4m3": 1e-6}
TC = ["fp16", "bf16", "e4m3", "tf32"]
GUARD = 64
SENT = complex(12345.0, -777.0)

# (r, M, K, L, F): tiny; the small FP32 case; ragged multi-tile; full lag K*L = N; a
# K = L = 1 degenerate; many K blocks and lag tiles
SHAPES = [(3, 1, 1, 1, 1), (7, 8, 2, 16, 1), (6, 3, 7, 9, 2), (10, 100, 5, 60, 3),
          (12, 64, 16, 128, 2), (5, 2, 31, 1, 1), (8, 65, 3, 85, 1)]


@pytest.fixture(scope="module")
def pk():
    import paper_2206_05506_gb300 as pk
    pk.lib()
    return pk


def _case(r, M, K, L, F, seed=0, snr=10.0):
    w = C.Workload("t", r=r, M=M, K=K, L=L, F=F, snr_db=(snr,), seed=seed)
    return C.make(w)


def _guarded(shape, dev):
    n = int(np.prod(shape))
    buf = torch.full((n + 2 * GUARD,), SENT, dtype=torch.complex64, device=dev)
    return buf, buf[GUARD:GUARD + n].view(*shape)


def _guards_ok(buf):
    g = torch.cat([buf[:GUARD], buf[-GUARD:]]).cpu().numpy()
    return bool(np.all(g == np.complex64(SENT)))


def _run(pk, Y, bits, K, L, dtype):
    dev = torch.device("cuda", 0)
    pilot = pk.Pilot(bits, device=dev)
    F, M, N = Y.shape
    buf, H = _guarded((F, M, K, L), dev)
    pk.estimate(torch.from_numpy(Y).to(dev), pilot, K, L, dtype=dtype, out=H)
    assert pk.get_status(dev) == 0
    assert _guards_ok(buf), "write outside H"
    return H.cpu().numpy()


@pytest.mark.parametrize("shape", SHAPES)
def test_fp32_simt_matches_oracle(pk, shape):
    r, M, K, L, F = shape
    bits, _, Y = _case(*shape)
    H = _run(pk, Y, bits, K, L, "fp32")
    ref = O.estimate(Y, bits, K, L)
    assert O.nmse(H, ref) <= TOL["fp32"]
    assert np.abs(H - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("dtype", TC)
@pytest.mark.parametrize("shape", SHAPES)
def test_tensor_core_matches_oracle(pk, shape, dtype):
    r, M, K, L, F = shape
    bits, _, Y = _case(*shape, seed=r)
    H = _run(pk, Y, bits, K, L, dtype)
    ref = O.estimate(Y, bits, K, L)
    refq = O.estimate_quantized(Y, bits, K, L, dtype)
    assert O.nmse(H, refq) <= TOL_Q[dtype], "accumulation error beyond FP32"
    assert O.nmse(H, ref) <= TOL[dtype]


def _decode(q, dtype):
    q = q.cpu()
    if dtype == "fp16":
        return q.view(torch.float16).double().numpy()
    if dtype == "bf16":
        return q.view(torch.bfloat16).double().numpy()
    if dtype == "tf32":
        return q.view(torch.float32).double().numpy()
    return q.view(torch.float8_e4m3fn).double().numpy()


@pytest.mark.parametrize("dtype", TC)
@pytest.mark.parametrize("shape", [(7, 8, 2, 16, 1), (10, 33, 1, 1, 2), (4, 3, 1, 1, 1)])
def test_quantizer_bit_exact(pk, shape, dtype):
    r, M, K, L, F = shape
    bits, _, Y = _case(*shape, seed=5, snr=0.0)
    # spread the antennas' powers over decades so the scales differ
    Y = (Y * np.logspace(-3, 3, M, dtype=np.float32)[None, :, None]).astype(np.complex64)
    dev = torch.device("cuda", 0)
    res = pk.quantize(torch.from_numpy(Y).to(dev), dtype, want_power=True)
    Q, se = O.quantize(Y, dtype)
    N = Y.shape[2]
    A = F * M
    rows = _decode(res["q"], dtype)[:, :N]
    assert rows.shape[0] == 16 * ((A + 7) // 8)
    # groups of 8 antennas: real rows, then imaginary rows; padding rows zero
    a = np.arange(A)
    re_rows = 16 * (a // 8) + a % 8
    got = np.stack([rows[re_rows], rows[re_rows + 8]], axis=1)
    want = np.stack([Q.real, Q.imag], axis=-2).reshape(A, 2, N)
    assert np.array_equal(got, want)
    pad = np.setdiff1d(np.arange(rows.shape[0]), np.concatenate([re_rows, re_rows + 8]))
    assert np.all(rows[pad] == 0)
    assert np.array_equal(pk.operand_rows(A)[0].numpy(), re_rows)
    assert np.array_equal(res["exps"].cpu().numpy(), se.reshape(-1))
    fac = np.float32(1.0 / N) * np.ldexp(np.float32(1.0), -se.reshape(-1)).astype(np.float32)
    assert np.array_equal(res["factor"].cpu().numpy(), fac)
    pw = (np.abs(Y.astype(np.complex128)) ** 2).mean(axis=-1).reshape(-1)
    assert np.allclose(res["power"].cpu().numpy(), pw, rtol=1e-12, atol=0)


@pytest.mark.parametrize("dtype", TC)
def test_quantizer_non_finite_samples(pk, dtype):
    # samples that are not numbers are ordinary data here: a NaN part is left out of the
    # antenna's peak, an infinite part (or no number at all) gives scale 1, and each part
    # is then rounded as IEEE 754 prescribes (infinity for fp16 / bf16 / tf32, +-448 for
    # e4m3); an all-zero antenna gets scale 1 and zero codes
    rng = np.random.default_rng(21)
    N = 67                                       # ragged: 16 groups of 4 and a tail of 3
    M = 11                                       # a ragged second 8-antenna group
    Y = ((rng.standard_normal((1, M, N)) + 1j * rng.standard_normal((1, M, N))) * 0.3)
    Y = Y.astype(np.complex64)
    Y[0, 0, 5] = complex(1.0, np.inf)           # an infinite part: scale 1
    Y[0, 1, [0, 9, 66]] = complex(np.nan, 0.5)  # NaN parts left out of the peak
    Y[0, 1, 33] = complex(-0.75, np.nan)
    Y[0, 2, :] = complex(np.nan, np.nan)        # no number at all: scale 1
    Y[0, 3, 64] = complex(0.0, -np.inf)         # in the ragged tail
    Y[0, 4, :] = 0.0                            # all zero: scale 1
    Y[0, 5, :] *= np.float32(1e-30)             # tiny but finite: a large scale
    dev = torch.device("cuda", 0)
    res = pk.quantize(torch.from_numpy(Y).to(dev), dtype, want_power=True)
    Q, se = O.quantize(Y, dtype)
    t = O.SCALE_TARGET_EXP[dtype]
    if t is not None:
        peak1 = np.nanmax(np.abs(np.stack([Y[0, 1].real, Y[0, 1].imag])))
        assert list(se[0, :5]) == [0, t - int(np.frexp(np.float64(peak1))[1]), 0, 0, 0]
        assert se[0, 5] == 100                   # the clamp
    rows = _decode(res["q"], dtype)[:, :N]
    a = np.arange(M)
    re_rows = 16 * (a // 8) + a % 8
    got = np.stack([rows[re_rows], rows[re_rows + 8]], axis=1)
    want = np.stack([Q.real, Q.imag], axis=-2).reshape(M, 2, N)
    assert np.array_equal(got, want, equal_nan=True)   # NaN at the same places
    pad = np.setdiff1d(np.arange(rows.shape[0]), np.concatenate([re_rows, re_rows + 8]))
    assert np.all(rows[pad] == 0)
    assert np.array_equal(res["exps"].cpu().numpy(), se.reshape(-1))
    fac = np.float32(1.0 / N) * np.ldexp(np.float32(1.0), -se.reshape(-1)).astype(np.float32)
    assert np.array_equal(res["factor"].cpu().numpy(), fac)
    pw = (np.abs(Y.astype(np.complex128)) ** 2).mean(axis=-1).reshape(-1)
    assert np.allclose(res["power"].cpu().numpy(), pw, rtol=1e-12, atol=0, equal_nan=True)
    assert pk.get_status(dev) == 0


def test_tensor_core_staged_pilot_path(pk, monkeypatch):
    # the per-stage pilot generator (used when the resident list does not fit) on shapes
    # with several K blocks, lag tiles and a ragged row tile
    monkeypatch.setenv("PNCE_TC_STAGED_PILOT", "1")
    for shape in [(10, 100, 5, 60, 3), (12, 64, 16, 128, 2), (6, 3, 7, 9, 2)]:
        r, M, K, L, F = shape
        bits, _, Y = _case(*shape, seed=11)
        for dtype in TC:
            H = _run(pk, Y, bits, K, L, dtype)
            refq = O.estimate_quantized(Y, bits, K, L, dtype)
            assert O.nmse(H, refq) <= TOL_Q[dtype], (shape, dtype)


@pytest.mark.parametrize("dtype", ["fp32"] + TC)
def test_paper_scale_workload(pk, dtype):
    # 128 frames of M=64, N=1023, K=8, L=64 at SNR 0/10/20 dB
    w = C.PAPER_SCALE
    bits, h, Y = C.make(w)
    H = _run(pk, Y, bits, w.K, w.L, dtype)
    ref = O.estimate(Y, bits, w.K, w.L)
    assert O.nmse(H, ref) <= TOL[dtype]
    snr = w.frame_snr()
    for s in np.unique(snr):                     # each SNR of the sweep on its own
        f = snr == s
        assert O.nmse(H[f], ref[f]) <= TOL[dtype], s
    if dtype == "fp32":
        assert np.abs(H - ref).max() <= 1e-5 * np.abs(ref).max()
    else:                                        # the accumulation, apart from rounding Y
        refq = O.estimate_quantized(Y, bits, w.K, w.L, dtype)
        assert O.nmse(H, refq) <= TOL_Q[dtype]
        per_frame = [O.nmse(H[i], refq[i]) for i in range(w.F)]
        assert max(per_frame) <= TOL_Q[dtype]


def test_noise_free_recovery_closed_form(pk):
    # Eq. 1-3: a noise-free block is estimated as h + (h - S)/N
    w = C.Workload("nf", r=10, M=16, K=8, L=64, F=2, snr_db=(0.0,), seed=4)
    bits, h, Y = C.make(w, noise=False)
    N = w.N
    x = h.reshape(w.F, w.M, -1)
    want = (x + (x - x.sum(-1, keepdims=True)) / N).reshape(h.shape)
    for dtype, tol in (("fp32", 1e-10), ("tf32", 1e-6), ("fp16", 1e-6)):
        H = _run(pk, Y, bits, w.K, w.L, dtype)
        assert O.nmse(H, want) <= tol, dtype


def test_real_pilot_forward_and_adjoint(pk):
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(1)
    # shapes: N below a warp's width and the degenerate N = 2; several 128-lag chunks and
    # 256-output tiles; more antennas than the dp grid's warps per tile (1500 at N = 511)
    for (F, M, N, K, L) in [(2, 3, 31, 2, 5), (3, 40, 1023, 8, 64), (1, 5, 300, 3, 100),
                            (1, 1, 7, 1, 7), (1, 2, 2, 1, 2), (3, 500, 511, 2, 128),
                            (1, 40, 4095, 16, 128)]:
        Y = (rng.standard_normal((F, M, N)) + 1j * rng.standard_normal((F, M, N))).astype(np.complex64)
        p = np.tanh(rng.standard_normal(N)).astype(np.float32)
        G = (rng.standard_normal((F, M, K, L)) + 1j * rng.standard_normal((F, M, K, L))).astype(np.complex64)
        Yd, pd, Gd = (torch.from_numpy(a).to(dev) for a in (Y, p, G))
        H = pk.estimate_real_pilot(Yd, pd, K, L).cpu().numpy()
        assert O.nmse(H, O.estimate_real_pilot(Y, p.astype(np.float64), K, L)) <= 1e-10
        dY, dp = pk.backward(pd, Yd, Gd, K, L)
        rdY, rdp = O.adjoint(G, Y, p.astype(np.float64), K, L)
        assert O.nmse(dY.cpu().numpy(), rdY) <= 1e-10
        assert O.nmse(dp.cpu().numpy(), rdp) <= 1e-10
        # deterministic: a second run is bitwise identical
        dY2, dp2 = pk.backward(pd, Yd, Gd, K, L)
        assert torch.equal(dp, dp2) and torch.equal(dY, dY2)


def test_deterministic_and_independent_of_batch(pk):
    # results per frame do not depend on the other frames of the launch
    bits, _, Y = _case(10, 64, 8, 64, 6, seed=8)
    dev = torch.device("cuda", 0)
    pilot = pk.Pilot(bits, device=dev)
    Yd = torch.from_numpy(Y).to(dev)
    for dtype in ["fp32"] + TC:
        full = pk.estimate(Yd, pilot, 8, 64, dtype=dtype)
        again = pk.estimate(Yd, pilot, 8, 64, dtype=dtype)
        part = pk.estimate(Yd[2:5].contiguous(), pilot, 8, 64, dtype=dtype)
        assert torch.equal(full, again)
        assert torch.equal(full[2:5], part)


def test_invalid_arguments(pk):
    dev = torch.device("cuda", 0)
    bits, _, Y = _case(7, 4, 2, 16, 1)
    pilot = pk.Pilot(bits, device=dev)
    Yd = torch.from_numpy(Y).to(dev)
    with pytest.raises(pk.PnceError) as e:
        pk.estimate(Yd, pilot, 8, 16)                       # K*L > N (Eq. 7)
    assert e.value.status == 1
    flat = torch.zeros(Y.size + 1, dtype=torch.complex64, device=dev)
    mis = flat[1:].view(Y.shape)                            # 8-byte aligned only
    with pytest.raises(pk.PnceError) as e:
        pk.estimate(mis, pilot, 2, 16)
    assert e.value.status == 1
    other = pk.Pilot(bits[:63], device=dev)
    lib = pk.lib()
    H = torch.empty((1, 4, 2, 16), dtype=torch.complex64, device=dev)
    st = lib.pnce_estimate(other.ctx.handle, other.handle, Yd.data_ptr(), 1, 4, 127, 2, 16, 0,
                           None, 0, H.data_ptr(), None)
    assert st == 6                                          # pilot length mismatch
    ws = torch.empty(16, dtype=torch.uint8, device=dev)
    st = lib.pnce_estimate(pilot.ctx.handle, pilot.handle, Yd.data_ptr(), 1, 4, 127, 2, 16, 2,
                           ws.data_ptr(), 16, H.data_ptr(), None)
    assert st == 1                                          # workspace too small
    assert pk.get_status(dev) == 0


@pytest.mark.parametrize("dtype", TC)
def test_long_sequence_staged_pilot(pk, dtype):
    # N = 16383: the pilot list of all K blocks no longer fits beside the pipeline, so the
    # kernel takes the per-stage pilot generator on its own (256 K blocks of fp16)
    r, M, K, L, F = 14, 9, 4, 256, 1
    bits, _, Y = _case(r, M, K, L, F, seed=2)
    H = _run(pk, Y, bits, K, L, dtype)
    refq = O.estimate_quantized(Y, bits, K, L, dtype)
    assert O.nmse(H, refq) <= TOL_Q[dtype]


def test_bad_output_buffers_rejected(pk):
    # a too-small, strided, host or wrong-dtype `out` is refused before any launch, and
    # the buffer it names is left as it was
    bits, _, Y = _case(7, 8, 2, 16, 1)
    dev = torch.device("cuda", 0)
    pilot = pk.Pilot(bits, device=dev)
    Yd = torch.from_numpy(Y).to(dev)
    small = torch.full((1, 8, 2, 15), SENT, dtype=torch.complex64, device=dev)
    for out in [small,
                torch.empty((1, 8, 2, 16), dtype=torch.complex64),             # host memory
                torch.empty((1, 8, 16, 2), dtype=torch.complex64, device=dev).transpose(2, 3),
                torch.empty((1, 8, 2, 16), dtype=torch.complex128, device=dev)]:
        for dtype in ("fp32", "fp16"):
            with pytest.raises(ValueError):
                pk.estimate(Yd, pilot, 2, 16, dtype=dtype, out=out)
    with pytest.raises(ValueError):                  # a workspace that is too small
        pk.estimate(Yd, pilot, 2, 16, dtype="fp16",
                    workspace=torch.empty(16, dtype=torch.uint8, device=dev))
    p = torch.zeros(127, dtype=torch.float32, device=dev)
    G = torch.zeros((1, 8, 2, 16), dtype=torch.complex64, device=dev)
    with pytest.raises(ValueError):                  # the pilot of the adjoint is checked
        pk.backward(p[:100], Yd, G, 2, 16)
    torch.cuda.synchronize()
    assert bool((small == SENT).all())
    assert pk.get_status(dev) == 0


def test_auto_dtype_follows_its_rule(pk):
    # dtype "auto": the same bits as the FP32 path at <= 16 lags and as fp16 above
    dev = torch.device("cuda", 0)
    for shape in [(10, 9, 2, 8, 2), (10, 9, 1, 16, 2), (10, 9, 1, 17, 2), (10, 9, 8, 64, 2)]:
        r, M, K, L, F = shape
        bits, _, Y = _case(*shape, seed=3)
        want = "fp32" if K * L <= 16 else "fp16"
        Yd = torch.from_numpy(Y).to(dev)
        pilot = pk.Pilot(bits, device=dev)
        Ha = pk.estimate(Yd, pilot, K, L, dtype="auto")
        Hw = pk.estimate(Yd, pilot, K, L, dtype=want)
        assert torch.equal(Ha, Hw), shape
        Hh = pk.estimate_host(torch.from_numpy(Y).pin_memory(), pilot, K, L, dtype="auto")
        assert torch.equal(Hh, Hw.cpu()), shape
    assert pk.get_status(dev) == 0


@pytest.mark.parametrize("KL", [1, 7, 16, 32])
def test_few_lags_result_independent_of_row_placement(pk, KL):
    # the few-lags FP32 kernel reads rows of odd N that alternately start on and half-way
    # into a 16-byte boundary; a row shifted by one position in the batch (so its start
    # flips between the two) must give the same bits, for even and odd N
    dev = torch.device("cuda", 0)
    for r in (6, 9):
        bits, _, Y = _case(r, 5, 1, KL, 2, seed=4)
        F, M, N = Y.shape
        pilot = pk.Pilot(bits, device=dev)
        Yd = torch.from_numpy(Y).to(dev)
        H = pk.estimate(Yd, pilot, 1, KL, dtype="fp32")
        Y2 = torch.cat([torch.zeros((1, 1, N), dtype=torch.complex64, device=dev),
                        Yd.reshape(1, F * M, N)], dim=1)
        H2 = pk.estimate(Y2, pilot, 1, KL, dtype="fp32").reshape(F * M + 1, 1, KL)
        assert torch.equal(H2[1:], H.reshape(F * M, 1, KL))
        assert O.nmse(H.cpu().numpy(), O.estimate(Y, bits, 1, KL)) <= 1e-10
