"""Writes the descriptor scaler table paper_2305_08140_gb300/data/q_scaler.json.

For each parameter seed, s_nu = 1 / max_i |q_nu^i| over the 2,000-atom c1
structure, with q computed by the FP64 oracle only.  The scaler plays the part
of NEP's per-component descriptor normalisation: random weights U(-0.5, 0.5)
applied to unscaled descriptors would leave some components negligible and
others large.

Run:  python -m oracle.make_scaler
"""
import json
import os

import numpy as np

from oracle import oracle as O
from paper_2305_08140_gb300 import inputs as I

SEEDS = (1, 101)


def main():
    s = I.c1()
    table = {"definition": "s_nu = 1 / max_i |q_nu^i| over the c1 structure "
                           "(2,000-atom bcc W, sigma 0.05 A, seed 0), q from the FP64 oracle",
             "scalers": {}}
    for seed in SEEDS:
        m = I.nep_model(seed, with_scaler=False)
        q = O.descriptors(m, s.pos, s.box, s.pbc)
        table["scalers"][str(seed)] = [float(v) for v in 1.0 / np.max(np.abs(q), axis=0)]
    out = os.path.join(os.path.dirname(I.__file__), "data", "q_scaler.json")
    with open(out, "w") as f:
        json.dump(table, f, indent=1)
    print("wrote", out)


if __name__ == "__main__":
    main()
