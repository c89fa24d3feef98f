"""Pilot-slot layouts on the GPU (Sec. II-A/B): received rows that still carry the cyclic
prefix, and the even-spread shift rule of Eq. 8, for every arithmetic, against the
oracle's general estimator on blocks produced by a linear channel acting on the
CP-prefixed pilot."""
import numpy as np
import pytest
import torch

from oracle import pn_oracle as O
from synth import channel as C
from synth import mseq

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-6, "tf32": 1e-6, "fp16": 2e-3, "bf16": 2e-3, "e4m3": 3e-2}

# (r, M, K, L, cp, F): small, ragged antenna count, odd L, L above one 256-lag tile,
# the Fig. 5 setup (PN 2047, N_batch 4, L = C = 128)
CASES = [(7, 3, 3, 20, 20, 2), (10, 37, 4, 100, 100, 2), (9, 5, 3, 45, 50, 1),
         (11, 4, 3, 300, 300, 1), (11, 16, 4, 128, 128, 4)]


def _case(r, M, K, L, cp, F, rule, seed=0, snr=10.0, noise=True):
    bits = mseq.mseq_bits(r, seed)
    N = bits.size
    rng = np.random.default_rng([seed, r, M, K, L, cp])
    h = C.channel(rng, F, M, K, L)
    sh = (C.shifts_kl if rule == "kl" else C.shifts_spread)(K, L, N)
    Y = C.received_with_cp(h, bits, snr, rng, cp, shifts=sh, noise=noise)
    return bits, h, Y, sh


@pytest.mark.parametrize("dtype", ["fp32", "fp16", "e4m3", "tf32"])
@pytest.mark.parametrize("rule", ["kl", "spread"])
@pytest.mark.parametrize("case", CASES)
def test_layout_matches_oracle(case, rule, dtype):
    import paper_2206_05506_gb300 as pk
    r, M, K, L, cp, F = case
    if rule == "kl" and K * L > (1 << r) - 1:
        pytest.skip("K*L > N")
    bits, h, Y, sh = _case(r, M, K, L, cp, F, rule)
    dev = torch.device("cuda", 0)
    pilot = pk.Pilot(bits, device=dev)
    n = F * M * K * L
    buf = torch.full((n + 64,), complex(9.0, 9.0), dtype=torch.complex64, device=dev)
    H = buf[32:32 + n].view(F, M, K, L)
    pk.estimate(torch.from_numpy(Y).to(dev), pilot, K, L, dtype=dtype, out=H, cp_len=cp,
                shift_rule=rule)
    assert pk.get_status(dev) == 0
    g = torch.cat([buf[:32], buf[-32:]]).cpu().numpy()
    assert np.all(g == np.complex64(complex(9.0, 9.0))), "write outside H"
    ref = O.estimate_general(Y, bits, K, L, cp_len=cp, shifts=sh)
    assert O.nmse(H.cpu().numpy(), ref) <= TOL[dtype]


def test_layout_noise_free_closed_form():
    import paper_2206_05506_gb300 as pk
    r, M, K, L, cp, F = 11, 16, 4, 128, 128, 2
    bits, h, Y, sh = _case(r, M, K, L, cp, F, "spread", noise=False)
    N = bits.size
    dev = torch.device("cuda", 0)
    pilot = pk.Pilot(bits, device=dev)
    x = h.reshape(F, M, K * L)
    want = (x + (x - x.sum(-1, keepdims=True)) / N).reshape(h.shape)
    for dtype, tol in (("fp32", 1e-10), ("fp16", 1e-6)):
        H = pk.estimate(torch.from_numpy(Y).to(dev), pilot, K, L, dtype=dtype, cp_len=cp,
                        shift_rule="spread")
        assert O.nmse(H.cpu().numpy(), want) <= tol


def test_layout_rejects_aliasing():
    import paper_2206_05506_gb300 as pk
    dev = torch.device("cuda", 0)
    bits = mseq.mseq_bits(7, 0)
    pilot = pk.Pilot(bits, device=dev)
    Y = torch.zeros((1, 2, 127 + 8), dtype=torch.complex64, device=dev)
    with pytest.raises(pk.PnceError) as e:
        pk.estimate(Y, pilot, 4, 40, cp_len=8, shift_rule="spread")    # 40 > 127 // 4
    assert e.value.status == 1


@pytest.mark.parametrize("dtype", ["fp16", "bf16", "e4m3", "tf32"])
def test_spread_kernels_agree(dtype, monkeypatch):
    # the even-spread tiles of 128 lags or fewer go to the lag-major kernel (CTA pairs on
    # the 2-SM MMA, or single CTAs); every form gives the same bits as the lag-column
    # kernel, across several row blocks, a ragged antenna count and an odd number of lag
    # tiles (no pairs)
    import paper_2206_05506_gb300 as pk
    dev = torch.device("cuda", 0)
    for (r, M, K, L, cp, F) in [(11, 37, 4, 128, 0, 5), (11, 16, 6, 100, 0, 9),
                                (12, 130, 16, 128, 0, 3), (10, 64, 3, 64, 64, 4)]:
        bits, h, Y, sh = _case(r, M, K, L, cp, F, "spread")
        pilot = pk.Pilot(bits, device=dev)
        Yd = torch.from_numpy(Y).to(dev)
        outs = []
        for lm, cl in (("0", ""), ("1", "1"), ("1", "")):
            monkeypatch.setenv("PNCE_TC_LAGMAJOR", lm)
            monkeypatch.setenv("PNCE_TC_LAGMAJOR_CL", cl)
            outs.append(pk.estimate(Yd, pilot, K, L, dtype=dtype, cp_len=cp,
                                    shift_rule="spread"))
        assert pk.get_status(dev) == 0
        for i in (1, 2):
            assert torch.equal(outs[0], outs[i]), (r, M, K, L, i)
        ref = O.estimate_general(Y, bits, K, L, cp_len=cp, shifts=sh)
        assert O.nmse(outs[2].cpu().numpy(), ref) <= TOL[dtype]
