"""The paper's experiments (Sec. IV) reduced in size, run through the library, and the
paper's qualitative findings asserted on what they give: MAE falls with the PN length and
its high-SNR floor rises with N_batch (Fig. 4, Eq. 12), the fp16 tensor-core MAE equals the
FP32 path's to 3 digits (Fig. 5), and every frame is estimated within its propagation time
at a 10 MHz sampling rate (Figs. 6 and 7, Eq. 11)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_paper_findings_hold():
    import paper_2206_05506_gb300 as pk
    import paper_experiments as PE

    dev = torch.device("cuda", 0)
    res = PE.run(pk, dev, "fp16", iters=6, snrs=[-10.0, 10.0, 40.0])
    c = PE.claims(res)
    assert c == {"mae_falls_with_pn_length": True, "floor_rises_with_n_batch": True,
                 "fp16_equals_fp32": True, "realtime_at_10MHz": True}, (c, res)
    assert pk.get_status(dev) == 0
