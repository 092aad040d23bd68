"""The settings the paper prints for the filtering / reconstruction fit
(tests/golden/paper_settings.json, Sec. IV-A and V-B) against the library's
defaults and the synthetic workloads."""
import json
import os

import pytest

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_settings.json")


def test_reconstruction_defaults_match_the_paper():
    from paper_2412_16750_gb300 import api, synth
    g = json.load(open(GOLDEN))
    names = g["params_order"]                      # the library's order v0, T, s0, a_max, b
    assert tuple(api.RECON_INIT[:5]) == tuple(g["init"][n] for n in names)
    assert tuple(api.RECON_BOX_LO) == tuple(g["bounds"][n][0] for n in names)
    assert tuple(api.RECON_BOX_HI) == tuple(g["bounds"][n][1] for n in names)
    assert (api.RECON_DP0, api.RECON_DV0) == (g["virtual_leader_init"]["dp"], g["virtual_leader_init"]["dv"])
    assert synth.A_MIN == g["a_min"]
    assert synth.FILTER_SPEC["dt"] == g["dt"]["filtering"]
    assert synth.RECON_SPEC["dt"] == g["dt"]["reconstruction"]
    # the fit's defaults: 500 Adam steps, lr 0.1 -> 0.01
    import inspect
    sig = inspect.signature(api.Recon.fit)
    assert sig.parameters["n_iter"].default == g["adam_steps"]
    assert (sig.parameters["lr0"].default, sig.parameters["lr1"].default) == tuple(g["lr"])
    # the zero-knowledge start of the coupled fit is the same point
    assert tuple(synth.PLAIN_INIT) == tuple(api.RECON_INIT)
