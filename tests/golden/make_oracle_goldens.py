"""Writes the stored oracle results used by the full-size GPU parity tests.

Calls only the oracle (and the input generator): the expected values never come
from the CUDA path.  Each file records a SHA-256 of the generated cohort, so a
test can tell when the generator produced a different cohort on another machine
and recompute the oracle live instead (or skip, where a live run would take
hours).

    python tests/golden/make_oracle_goldens.py            # every workload
    python tests/golden/make_oracle_goldens.py c3_r2 ...  # only the named ones

The h = 4 workloads at full sample width take the single-threaded oracle from
minutes (c3w_pdfs) to hours (c3_r2: the first two greedy rounds of the full
19,000-gene cohort), so they are written once, offline, and kept.
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

WORKLOADS = {
    # name: (cohort spec, h, alpha, max_rounds)
    "c2_pdfs": (synth.c2(), 3, (1, 10), -1),
    "c1_pdfs": (synth.c1(), 2, (1, 10), -1),
    # the full h = 4 workload (G=19,000, Nt=800, Nn=400, 128-bit rows): first rounds only
    "c3_r2": (synth.c3(), 4, (1, 10), 2),
    # the same law and sample width (14 tumor words, 7 normal words) at G = 5,000: whole solve
    "c3w_pdfs": (synth.c3_law(5000, 800, 400, 3), 4, (1, 10), -1),
}


def cohort_hash(bitmaps) -> str:
    return hashlib.sha256(bitmaps.tobytes()).hexdigest()


def solve(name):
    spec, h, alpha, max_rounds = WORKLOADS[name]
    c = synth.generate(spec)
    t = time.time()
    sol = oracle.pdfs(c.bitmaps, c.G, c.Nt, c.Nn, h, alpha, max_rounds=max_rounds)
    dt = time.time() - t
    return {
        "workload": name, "G": c.G, "Nt": c.Nt, "Nn": c.Nn, "h": h, "alpha": list(alpha), "seed": spec.seed,
        "max_rounds": max_rounds,
        "cohort_sha256": cohort_hash(c.bitmaps),
        "records": [[list(g), tp, fp] for g, tp, fp in sol.records()],
        "visited": sol.visited.astype(int).tolist(), "pruned": sol.pruned.astype(int).tolist(),
        "oracle_seconds": round(dt, 2),
    }


def main(names):
    for name in names or list(WORKLOADS):
        out = solve(name)
        with open(os.path.join(HERE, f"{name}.json"), "w") as f:
            json.dump(out, f, separators=(",", ":"))
        print(name, "k =", len(out["records"]), "rounds =", len(out["visited"]), f"{out['oracle_seconds']} s",
              flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
