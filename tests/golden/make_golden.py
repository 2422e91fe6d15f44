"""Writes oracle_small_runs.json: the FP64 oracle's own results on two small
seeded Big-means runs (Alg. 1, then the final assignment of Sec. 3.4).

This is a regression record, not a pin.  It makes any later change of the
oracle's arithmetic show up as a changed file, and
tests/test_oracle.py::test_oracle_reproduces_its_recorded_runs compares
against it.  The script calls only ``oracle`` and the seeded input generators
of ``bminputs``.  Run it from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import bminputs as bi  # noqa: E402
import oracle as o  # noqa: E402

# (name, m, n, k, s, chunks, components, seed, box)
CASES = [("blobs_2d_m400_k4", 400, 2, 4, 120, 4, 5, 3, 8.0),
         ("blobs_5d_m600_k6", 600, 5, 6, 200, 3, 7, 11, 5.0)]


def run(m, n, k, s, chunks, comps, seed, box):
    X, _ = bi.mixtures.isotropic_blobs(m, n, comps, seed, box=box)
    draws = [bi.chunk_draws(seed, t, m, s, k) for t in range(chunks)]
    st, recs = o.big_means(X, k, draws)
    labels, sse, _, _ = o.final_assignment(X, st.C.astype(np.float32), st.live)
    return {"f_opt": st.f_opt, "C": st.C.tolist(), "live": st.live.astype(int).tolist(),
            "sse": sse, "labels_sum": int(np.asarray(labels, np.int64).sum()),
            "accepted": [bool(r.accepted) for r in recs],
            "iters": [int(r.iters) for r in recs]}


def main():
    out = {"about": "FP64 oracle results on small seeded runs (regression record, "
                    "written by tests/golden/make_golden.py from oracle/ only)",
           "cases": []}
    for name, m, n, k, s, chunks, comps, seed, box in CASES:
        rec = dict(name=name, m=m, n=n, k=k, s=s, chunks=chunks, components=comps,
                   seed=seed, box=box)
        rec["result"] = run(m, n, k, s, chunks, comps, seed, box)
        out["cases"].append(rec)
    with open(os.path.join(HERE, "oracle_small_runs.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
