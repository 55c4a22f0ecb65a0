"""Writes the descriptor scaler table paper_2305_08140_gb300/data/q_scaler.json.

For each parameter seed, s_nu = 1 / max |q_nu^i| over every atom i of the
scaler structures (c1 crystal, hot crystal, liquid-like packing, compressed
crystal -- the kinds of structure in the paper's W training set, Sec. III.A),
with q computed by the FP64 oracle only.  The scaler plays the part of NEP's
per-component descriptor normalisation: random weights U(-0.5, 0.5) applied to
unscaled descriptors would leave some components negligible and others large.

Run:  python -m oracle.make_scaler
"""
import json
import os

import numpy as np

from oracle import oracle as O
from paper_2305_08140_gb300 import inputs as I

MODELS = ((1, ("W",)), (101, ("W",)), (301, ("W", "Mo")), (401, ("W", "Mo", "Ta", "Nb")))


def main():
    table = {"definition": "s_nu = 1 / max |q_nu^i| over all atoms of inputs.scaler_structures() "
                           "(c1 crystal; 432-atom crystal sigma 0.3 A; 128-atom liquid-like "
                           "packing; 432-atom crystal at 0.9 a, sigma 0.1 A; for several "
                           "species, equiatomic random solid solutions of them); q from the "
                           "FP64 oracle; key 'seed' (W) or 'seed:species'",
             "scalers": {}}
    for seed, species in MODELS:
        m = I.nep_model(seed, with_scaler=False, species=species)
        qmax = np.zeros(m.dim)
        for s in I.scaler_structures(m.n_types):
            q = O.descriptors(m, s.pos, s.box, s.pbc, use_grid=False, types=s.types)
            qmax = np.maximum(qmax, np.max(np.abs(q), axis=0))
        table["scalers"][I.scaler_key(seed, species)] = [float(v) for v in 1.0 / qmax]
    out = os.path.join(os.path.dirname(I.__file__), "data", "q_scaler.json")
    with open(out, "w") as f:
        json.dump(table, f, indent=1)
    print("wrote", out)


if __name__ == "__main__":
    main()
