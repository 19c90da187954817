"""Reader of the hand-derived fixtures in tests/golden/hand_cases.txt."""
import os
from dataclasses import dataclass, field

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@dataclass
class HandCase:
    name: str
    G: int
    Nt: int
    Nn: int
    h: int
    alpha: tuple
    tumors: dict = field(default_factory=dict)   # gene -> list of tumor samples
    normals: dict = field(default_factory=dict)  # gene -> list of normal samples
    expect: list = field(default_factory=list)   # [(tuple, tp, fp)]

    def bitmaps(self) -> np.ndarray:
        Wt, Wn = (self.Nt + 63) // 64, (self.Nn + 63) // 64
        bm = np.zeros((self.G, Wt + Wn), dtype=np.uint64)
        for g in range(self.G):
            for s in self.tumors.get(g, []):
                bm[g, s // 64] |= np.uint64(1 << (s % 64))
            for s in self.normals.get(g, []):
                bm[g, Wt + s // 64] |= np.uint64(1 << (s % 64))
        return bm


def _samples(tok):
    if tok == "-":
        return []
    out = []
    for part in tok.split(","):
        if "-" in part:
            a, b = part.split("-")
            out.extend(range(int(a), int(b) + 1))
        else:
            out.append(int(part))
    return out


def load_hand_cases(path=None):
    path = path or os.path.join(GOLDEN, "hand_cases.txt")
    cases, cur = [], None
    with open(path) as f:
        for raw in f:
            line = raw.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "case":
                cur = HandCase(tok[1], 0, 0, 0, 0, (1, 1))
            elif tok[0] == "dims":
                G, Nt, Nn, h, an, ad = map(int, tok[1:7])
                cur.G, cur.Nt, cur.Nn, cur.h, cur.alpha = G, Nt, Nn, h, (an, ad)
            elif tok[0] == "gene":
                g = int(tok[1])
                assert tok[2] == "T" and tok[4] == "N"
                cur.tumors[g] = _samples(tok[3])
                cur.normals[g] = _samples(tok[5])
            elif tok[0] == "expect":
                genes = tuple(int(x) for x in tok[1].strip("()").split(",") if x)
                cur.expect.append((genes, int(tok[2]), int(tok[3])))
            elif tok[0] == "end":
                cases.append(cur)
                cur = None
    return cases
