"""Host-side check of the paper-experiment claims: tables that break each of the paper's
qualitative findings are caught, so the GPU test's assertions are not vacuous."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_claims_detect_a_violation():
    # the checks are not vacuous: tables that break each finding are caught (host only)
    import paper_experiments as PE

    good = {"fig4": {"pn511_nb1": [0.12, 0.004], "pn511_nb2": [0.12, 0.005],
                     "pn511_nb4": [0.12, 0.006], "pn2047_nb1": [0.06, 0.001],
                     "pn2047_nb2": [0.06, 0.002], "pn2047_nb4": [0.06, 0.003]},
            "fig5": {"lnz1": [0.0620, 0.0010]}, "fig5_fp32": {"lnz1": [0.0620, 0.0010]},
            "fig6": {"pn511": [{"realtime_at_10MHz": True}]}}
    assert all(PE.claims(good).values())
    bad = {k: (dict(v) if isinstance(v, dict) else v) for k, v in good.items()}
    bad["fig4"] = dict(good["fig4"], pn2047_nb4=[0.13, 0.003])
    assert not PE.claims(bad)["mae_falls_with_pn_length"]
    bad["fig4"] = dict(good["fig4"], pn511_nb4=[0.12, 0.0045])
    assert not PE.claims(bad)["floor_rises_with_n_batch"]
    bad["fig5"] = {"lnz1": [0.0622, 0.0010]}
    assert not PE.claims(bad)["fp16_equals_fp32"]
    bad["fig6"] = {"pn511": [{"realtime_at_10MHz": False}]}
    assert not PE.claims(bad)["realtime_at_10MHz"]
