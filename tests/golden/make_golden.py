"""Writes the stored expected values that are not printed in the paper.

Calls only the oracle (exact diagonalisation on the 4x4 torus); run from the
repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ed  # noqa: E402


def main():
    out = {"_source": "oracle.ed.tfim_ground_energy: Lanczos on the 2^16 space of the 4x4 torus"}
    for h in (2.0, 5.0):
        out["tfim_4x4_e_site_h%.1f" % h] = ed.tfim_ground_energy(4, 4, h)
    with open(os.path.join(HERE, "ed_4x4.json"), "w") as f:
        json.dump(out, f, indent=2)


if __name__ == "__main__":
    main()
