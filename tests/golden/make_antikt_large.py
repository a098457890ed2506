"""Writes tests/golden/antikt_large_r04.json: the FP64 oracle's anti-kt jets (R = 0.4)
of one large synthetic event, for the GPU parity test of an event of more than 5,000
particles (7,500 elements, 5,201 particles; the oracle's plain O(N^3) clustering takes
about 20 minutes on it, too long to run inside the test).  Calls only oracle/ and synth/.

    PYTHONPATH=. python tests/golden/make_antikt_large.py
"""
import json
import os

import numpy as np

import synth
from oracle import jets as J

SEED_EVENTS, SEED_TARGETS, SIZE, R = 45, 46, 7500, 0.4
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "antikt_large_r04.json")


def main():
    x, cu = synth.gen_events(SEED_EVENTS, [SIZE])
    cls, reg = synth.gen_targets(SEED_TARGETS, x, cu)
    jets, jof = J.event_jets(cls, reg, R)
    with open(OUT, "w") as f:
        json.dump({"what": f"FP64 oracle anti-kt jets of synth.gen_events({SEED_EVENTS}, [{SIZE}]) "
                           f"with synth.gen_targets({SEED_TARGETS}, ...) classes and regressions",
                   "seed_events": SEED_EVENTS, "seed_targets": SEED_TARGETS, "size": SIZE, "R": R,
                   "n_particles": int((jof >= 0).sum()),
                   "jet_of": jof.tolist(), "jets": np.round(jets, 9).tolist()}, f)


if __name__ == "__main__":
    main()
