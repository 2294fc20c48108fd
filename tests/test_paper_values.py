"""The numbers the paper prints (tests/golden/paper_printed_values.json, each with its
passage) against the oracle's constants and the library's defaults, independently.

The paper prints no worked example of its method, so these are its stated parameters:
the amplitudes of Eq. 1-4, the Table 1 bounds, the lean blend's phi, the time step and
the network widths of Sec. 3.2. A transcription slip on either side fails here. No GPU
compute: the library's defaults come from a host-only call.
"""
import inspect
import json
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_printed_values.json")


@pytest.fixture(scope="module")
def paper():
    with open(GOLDEN) as f:
        return json.load(f)


def test_every_value_cites_its_passage(paper):
    for k, v in paper.items():
        if k != "source":
            assert v["cite"].startswith("Sec. "), k


def test_oracle_hfrd_constants(paper):
    from oracle import hfrd as H
    a = paper["hfrd_amplitudes"]
    assert (H.ALPHA, H.BETA, H.GAMMA) == (a["alpha"], a["beta"], a["gamma"])
    c = paper["hfrd_constraints"]
    assert H.HC_RANGE == tuple(c["hc_ratio"])
    assert H.ON_RANGE == tuple(c["on_ratio"])
    assert H.PHI_RANGE == tuple(c["phi"])
    phi = inspect.signature(H.adiabatic_equilibrium).parameters["phi"].default
    assert phi == paper["lean_blend_phi"]["value"]


def test_library_hfrd_defaults(paper):
    from paper_2312_05800_gb300 import binding, build
    build.build()                                  # (a no-op once the library is built)
    q = binding.hfrd_params()                      # chem_hfrd_params_default: host code only
    a, c = paper["hfrd_amplitudes"], paper["hfrd_constraints"]
    assert (q.alpha, q.beta, q.gamma) == (a["alpha"], a["beta"], a["gamma"])
    assert (q.hc_lo, q.hc_hi) == tuple(c["hc_ratio"])
    assert (q.on_lo, q.on_hi) == tuple(c["on_ratio"])
    assert (q.phi_lo, q.phi_hi) == tuple(c["phi"])


def test_step_and_network_defaults(paper):
    from paper_2312_05800_gb300 import train
    assert train.DT == paper["time_step_s"]["value"]
    phi = inspect.signature(train.lean_equilibrium).parameters["phi"].default
    assert phi == paper["lean_blend_phi"]["value"]
    import bench
    assert bench.DT == paper["time_step_s"]["value"]
    assert tuple(bench.HIDDEN["c2"]) == tuple(paper["hidden_layers"]["value"])
