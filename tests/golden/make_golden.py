"""Writes tests/golden/cfg1_oracle.json from the CPU oracle alone.

The stored numbers come from nothing but ``oracle/`` run on the seeded
Gamma-point two-centre workload (cubic 8 bohr cell, Cartesian s(10,1,0.2) +
p(1,0.3) per centre, omega 0.3, exp(-G^2/4w^2) > 1e-14, pair overlap >
1e-12).  They guard the oracle against unintended changes; the oracle's
correctness itself is pinned by tests/test_oracle_pins.py.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2509_16460_gb300 import workloads as W  # noqa: E402


def main():
    w = W.cfg1()
    r = oracle.lrj(w, nthreads=1)
    J = r["Jk"][0, 0].real
    picks = [(0, 0), (0, 5), (3, 12), (8, 17), (17, 17), (4, 9)]
    G = r["G"]
    gpick = [0, 17, 101, 200, len(G) - 1]
    out = dict(
        workload=w.name,
        source="oracle/oracle.c orc_lrj, FP64, 1 thread",
        nG=int(r["nG"]), npairs=int(r["npairs"]),
        EJ=float(r["EJ"][0]),
        J=[[i, j, float(J[i, j])] for i, j in picks],
        rho=[[int(G[g][0]), int(G[g][1]), int(G[g][2]), float(r["rho"][0, g].real), float(r["rho"][0, g].imag)]
             for g in gpick],
    )
    with open(os.path.join(HERE, "cfg1_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
