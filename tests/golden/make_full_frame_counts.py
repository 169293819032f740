"""Write full_frame_counts.txt: the FP64 oracle's work counts for the full-size
frame (seed 0: 32^3 -> 256^3 localization, 512^2 render).  Calls only the
seeded generator and oracle/.  Run from the repository root:
    python tests/golden/make_full_frame_counts.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import field, localize, render  # noqa: E402
from paper_2007_13988_gb300 import synth  # noqa: E402


def counts():
    w = synth.full(0)
    lv = localize.hierarchical(lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P),
                               w.n0, w.num_levels)
    _, hit, _ = render.first_crossing(lv[-1].values, w.render)
    out = {f"evals_level{i}": l.n_eval for i, l in enumerate(lv)}
    out.update({f"rounds_level{i}": l.conflict_rounds for i, l in enumerate(lv)})
    out["evals_total"] = sum(l.n_eval for l in lv)
    out["dense_evals_finest"] = (lv[-1].N + 1) ** 3
    out["hits"] = int(np.count_nonzero(hit))
    out["inside_finest"] = int(np.count_nonzero(lv[-1].binary))
    return out


if __name__ == "__main__":
    c = counts()
    with open(os.path.join(HERE, "full_frame_counts.txt"), "w") as fh:
        fh.write("# FP64 oracle work counts of the full-size frame (seed 0): 32^3 -> 256^3\n")
        fh.write("# localization (Sec. 3.2) and a 512^2 render; written by\n")
        fh.write("# tests/golden/make_full_frame_counts.py (generator + oracle only).\n")
        for k, v in c.items():
            fh.write(f"{k} = {v}\n")
    print(c)
