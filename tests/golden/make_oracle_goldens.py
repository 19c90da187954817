"""Writes the stored oracle results used by the full-size GPU parity tests.

Calls only the oracle (and the input generator): the expected values never come
from the CUDA path.  Each file records a SHA-256 of the generated cohort, so a
test can tell when the generator produced a different cohort on another machine
and recompute the oracle live instead.

    python tests/golden/make_oracle_goldens.py
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
    # name: (cohort spec, h, alpha)
    "c2_pdfs": (synth.c2(), 3, (1, 10)),
    "c1_pdfs": (synth.c1(), 2, (1, 10)),
}


def cohort_hash(bitmaps) -> str:
    return hashlib.sha256(bitmaps.tobytes()).hexdigest()


def solve(name):
    spec, h, alpha = WORKLOADS[name]
    c = synth.generate(spec)
    t = time.time()
    sol = oracle.pdfs(c.bitmaps, c.G, c.Nt, c.Nn, h, alpha)
    dt = time.time() - t
    return {
        "workload": name, "G": c.G, "Nt": c.Nt, "Nn": c.Nn, "h": h, "alpha": list(alpha), "seed": spec.seed,
        "cohort_sha256": cohort_hash(c.bitmaps),
        "records": [[list(g), tp, fp] for g, tp, fp in sol.records()],
        "visited": sol.visited.astype(int).tolist(), "pruned": sol.pruned.astype(int).tolist(),
        "oracle_seconds": round(dt, 2),
    }


def main():
    for name in WORKLOADS:
        out = solve(name)
        with open(os.path.join(HERE, f"{name}.json"), "w") as f:
            json.dump(out, f, separators=(",", ":"))
        print(name, "k =", len(out["records"]), "rounds =", len(out["visited"]), f"{out['oracle_seconds']} s")


if __name__ == "__main__":
    main()
