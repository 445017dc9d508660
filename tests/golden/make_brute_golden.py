"""Writes brute_tiny.json: T and t of the seeded cases in cases.py by the
40-digit matrix-exponential solve of oracle/brute.py (each slice's ODE
c'' = (H_p - E) c integrated exactly, V = 0 electrodes; no eigenmodes, no
S-matrices).  Only oracle/ computes; run from the repository root:
    python -m tests.golden.make_brute_golden"""
import json
import os

import numpy as np

from oracle import pw_oracle as O
from oracle.brute import brute_transmission
from tests.golden.cases import CASES, tiny_instance


def main():
    out = []
    for seed, E, k, nsl in CASES:
        inst, dz = tiny_instance(seed, E, k, nsl)
        m = O.Model(inst)
        Hs = [O.hamiltonian(m.mn, m.G, np.array(k), t, m.half) for t in m.tables]
        kg2 = ((m.G + np.array(k)) ** 2).sum(1)
        T, t = brute_transmission(Hs, dz, kg2, kg2, E, dps=40)
        out.append({"seed": seed, "E": E, "kpar": list(k), "slices": nsl, "T": float(T),
                    "t_re": np.real(t).tolist(), "t_im": np.imag(t).tolist(),
                    "open_kg2": sorted(float(x) for x in kg2 if x < E)})
    doc = {"what": "T and flux-normalised t (open right x open left, channels in G-list order) of "
                   "the slice model, Sec. II A / Eq. loc, by an independent 40-digit solve",
           "digits": 40, "cases": out}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "brute_tiny.json"), "w") as f:
        json.dump(doc, f, indent=1)


if __name__ == "__main__":
    main()
