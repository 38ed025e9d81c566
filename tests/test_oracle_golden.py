"""The oracle still reproduces its stored cfg1 snapshot (tests/golden/cfg1_oracle.json,
written by tests/golden/make_golden.py, which calls only the oracle)."""
import json
import os

import numpy as np

from paper_2509_16460_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def test_cfg1_snapshot(orc):
    with open(os.path.join(HERE, "golden", "cfg1_oracle.json")) as f:
        ref = json.load(f)
    w = W.cfg1()
    r = orc.lrj(w, nthreads=1)
    assert r["nG"] == ref["nG"] == 340
    assert r["npairs"] == ref["npairs"] == 1118
    assert abs(r["EJ"][0] - ref["EJ"]) < 1e-13
    J = r["Jk"][0, 0].real
    for i, j, v in ref["J"]:
        assert abs(J[i, j] - v) < 1e-13
    G = [tuple(g) for g in r["G"].tolist()]
    for n1, n2, n3, re, im in ref["rho"]:
        g = G.index((n1, n2, n3))
        assert abs(r["rho"][0, g] - (re + 1j * im)) < 1e-13
    assert np.isfinite(r["EJ"]).all()
