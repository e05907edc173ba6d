"""Writes small_oracle.json: the oracle's outputs on the small synthetic
workload (M=20, 5+5 electrons, 100 determinants, 60 Cholesky vectors,
16 walkers, seed 0). Calls only the oracle and the input generator.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2406_08314_gb300 import synth  # noqa: E402


def main():
    s, w = synth.config_system("small", seed=0)
    out = oracle.msd(s, w.phi_a, w.phi_b, energy=True, vbias=True)
    cp = lambda z: [[float(v.real), float(v.imag)] for v in z]
    doc = {
        "what": "oracle outputs, small synthetic workload, seed 0",
        "ovlp": cp(out["ovlp"]),
        "e_loc": cp(out["e_loc"]),
        "vbias_w0": cp(out["vbias"][0]),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "small_oracle.json")
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)


if __name__ == "__main__":
    main()
