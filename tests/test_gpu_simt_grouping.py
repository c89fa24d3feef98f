"""The FP32 SIMT correlation splits the rows of a large grid into balanced groups (fewer
than 32 rows per block) and keeps full 32-row groups for small grids; every output is
summed over the samples in the same order either way, so the results must be bitwise
identical.  Checked for the plain estimate, the real-pilot forward and the dY adjoint."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


# 6144 rows x 2 lag tiles and 8000 rows x 1 lag tile: both grids fill at least half of the
# resident blocks, so they are rebalanced; one frame's grid is not
@pytest.mark.parametrize("F, M, N, K, L", [(96, 64, 1023, 8, 64), (80, 100, 511, 4, 64)])
def test_large_grid_equals_frame_by_frame(F, M, N, K, L):
    import paper_2206_05506_gb300 as pk
    from synth import mseq
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(F * 7 + M)
    bits = mseq.mseq_bits(int(np.log2(N + 1)), seed=1)
    Y = (rng.standard_normal((F, M, N)) + 1j * rng.standard_normal((F, M, N))).astype(np.complex64)
    Yd = torch.from_numpy(Y).to(dev)
    pilot = pk.Pilot(bits, device=dev)
    theta = torch.from_numpy(rng.standard_normal(N).astype(np.float32)).to(dev)
    G = torch.from_numpy((rng.standard_normal((F, M, K, L))
                          + 1j * rng.standard_normal((F, M, K, L))).astype(np.complex64)).to(dev)

    H = pk.estimate(Yd, pilot, K, L, dtype="fp32")
    Hr = pk.estimate_real_pilot(Yd, theta, K, L, pilot_map="tanh")
    dY, _ = pk.backward(theta, Yd, G, K, L, need_dp=False, pilot_map="tanh")
    for f in range(F):
        y = Yd[f:f + 1].contiguous()
        assert torch.equal(pk.estimate(y, pilot, K, L, dtype="fp32"), H[f:f + 1])
        assert torch.equal(pk.estimate_real_pilot(y, theta, K, L, pilot_map="tanh"), Hr[f:f + 1])
        d1, _ = pk.backward(theta, y, G[f:f + 1].contiguous(), K, L, need_dp=False,
                            pilot_map="tanh")
        assert torch.equal(d1, dY[f:f + 1])
