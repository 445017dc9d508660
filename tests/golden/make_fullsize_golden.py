"""Writes oracle results at the workloads' full sizes, for parity tests that
the oracle cannot finish inside a test run:

  junction512_k5.json   T and (n_open^L, n_open^R) of all 128 energies at the
                        sixth k_par of the N_G = 512, 320-slice AB junction
                        (the call the benchmark times), App. C / Sec. II B
  junction401.json      T of four seeded points of the N_G = 401 (whole
                        shells, E_cut = 29.34 Ry), 240-slice AB junction
  uneven96.json         T of eight of the first 96 instances of the uneven
                        batch (the six with the least work n^3 (N_s + 1) and
                        the two with the least work among those of N_G >= 256)

Only oracle/ computes (Eq. loc eigenmodes, Eqs. transfer and scatter, Eq.
recurrence applied left to right, the flux-normalised t of App. C).  Each file
is rewritten after every point, so an interrupted run resumes where it
stopped.  Run from the repository root:
    python -m tests.golden.make_fullsize_golden junction512_k5
    python -m tests.golden.make_fullsize_golden junction401
    python -m tests.golden.make_fullsize_golden uneven96"""
import json
import os
import sys
import time

import numpy as np

from oracle import pw_oracle as O
from synthetic import junction, junction_ecut_for, uneven_batch

HERE = os.path.dirname(os.path.abspath(__file__))

# the four points of the N_G = 401 junction: (energy index, k_par index) of
# its 128 x 32 grid, drawn once with the stated seed
J401_POINTS_SEED = 1504_01462 + 2


def j401_points():
    rng = np.random.default_rng(J401_POINTS_SEED)
    e = rng.choice(128, size=4, replace=False)
    k = rng.choice(32, size=4, replace=False)
    return [(int(a), int(b)) for a, b in zip(e, k)]


def _load(path):
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return None


def _save(path, doc):
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(doc, f, indent=1)
    os.replace(tmp, path)


def _point(model, modes, E):
    EL, ER = modes[0][0], modes[-1][0]
    nop = [int(len(O.open_channels(E, EL))), int(len(O.open_channels(E, ER)))]
    if min(nop) == 0:
        return 0.0, nop        # t has no entries: an electrode carries no current at E
    S = model.total_s(modes, E)
    _, T = O.transmission_from_s(S, E, EL, ER)
    return T, nop


def junction512_k5():
    path = os.path.join(HERE, "junction512_k5.json")
    inst = junction(ng=512, n_slices=320, n_e=128, n_k=32)
    kk = 5
    idx = list(range(kk * 128, (kk + 1) * 128))
    doc = _load(path) or {
        "what": "oracle T(E, k_par) and open-channel counts (left, right) of the AB junction, "
                "N_G = 512 (first 512 G by (|G|^2, m, n)), 320 slices, at k_par index 5 of 32 "
                "and all 128 energies (point indices 640..767 of junction(ng=512, n_slices=320))",
        "k_index": kk, "kpar": [float(x) for x in inst.kpar[idx[0]]],
        "energies": [float(inst.energies[i]) for i in idx], "T": [None] * 128, "nopen": [None] * 128}
    model = O.Model(inst)
    modes = model.modes(inst.kpar[idx[0]])
    for j, i in enumerate(idx):
        if doc["T"][j] is not None:
            continue
        t0 = time.time()
        T, nop = _point(model, modes, float(inst.energies[i]))
        doc["T"][j], doc["nopen"][j] = T, nop
        _save(path, doc)
        print(f"junction512 k5 e{j}: T = {T:.15g} nopen {nop} ({time.time() - t0:.0f} s)", flush=True)


def junction401():
    path = os.path.join(HERE, "junction401.json")
    inst = junction(ng=0, ecut=junction_ecut_for(401), n_slices=240, n_e=128, n_k=32)
    pts = j401_points()
    doc = _load(path) or {
        "what": "oracle T(E, k_par) of the AB junction with whole shells |G|^2 <= 29.34 Ry "
                "(N_G = 401), 240 slices, at four seeded (energy, k_par) indices of its 128 x 32 grid",
        "seed": J401_POINTS_SEED, "points": pts,
        "energies": [float(inst.energies[k * 128 + e]) for e, k in pts],
        "kpar": [[float(x) for x in inst.kpar[k * 128 + e]] for e, k in pts],
        "T": [None] * len(pts), "nopen": [None] * len(pts)}
    model = O.Model(inst)
    assert model.n == 401
    for j, (e, k) in enumerate(pts):
        if doc["T"][j] is not None:
            continue
        t0 = time.time()
        i = k * 128 + e
        modes = model.modes(inst.kpar[i])
        T, nop = _point(model, modes, float(inst.energies[i]))
        doc["T"][j], doc["nopen"][j] = T, nop
        _save(path, doc)
        print(f"junction401 point {j}: T = {T:.15g} nopen {nop} ({time.time() - t0:.0f} s)", flush=True)


def uneven96_picks(insts):
    """Indices (into the first 96 instances) of the stored uneven points."""
    work = [float(x.ng_exact) ** 3 * (x.n_slices + 1) for x in insts]
    order = sorted(range(len(insts)), key=lambda i: work[i])
    small = order[:6]
    big = [i for i in order if insts[i].ng_exact >= 256 and i not in small][:2]
    return sorted(small + big)


def uneven96():
    path = os.path.join(HERE, "uneven96.json")
    insts = uneven_batch(2048)[:96]
    picks = uneven96_picks(insts)
    doc = _load(path) or {
        "what": "oracle T of instances of uneven_batch(2048)[:96] (one (E, k_par) point each)",
        "index": picks, "ng": [insts[i].ng_exact for i in picks], "slices": [insts[i].n_slices for i in picks],
        "T": [None] * len(picks), "nopen": [None] * len(picks)}
    for j, i in enumerate(picks):
        if doc["T"][j] is not None:
            continue
        t0 = time.time()
        x = insts[i]
        model = O.Model(x)
        modes = model.modes(x.kpar[0])
        T, nop = _point(model, modes, float(x.energies[0]))
        doc["T"][j], doc["nopen"][j] = T, nop
        _save(path, doc)
        print(f"uneven96 instance {i} (N_G {x.ng_exact}, {x.n_slices} slices): T = {T:.15g} "
              f"({time.time() - t0:.0f} s)", flush=True)


if __name__ == "__main__":
    for what in sys.argv[1:] or ["junction401", "junction512_k5"]:
        {"junction512_k5": junction512_k5, "junction401": junction401, "uneven96": uneven96}[what]()
