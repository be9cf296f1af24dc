"""Edge lists for the closed-form fixtures in closed_forms.json."""
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load():
    spec = json.load(open(os.path.join(HERE, "closed_forms.json")))
    out = []
    for g in spec["graphs"]:
        n, fam, W = g["n"], g["family"], g["weights"]
        e = []
        if fam == "path":
            e = [(i, i + 1, W[i]) for i in range(n - 1)]
        elif fam == "cycle":
            e = [(i, (i + 1) % n, W) for i in range(n)]
        elif fam == "cycle_heavy":
            e = [(i, (i + 1) % n, W) for i in range(n - 1)] + [(n - 1, 0, g["heavy"])]
        elif fam == "star":
            e = [(0, i + 1, W[i]) for i in range(n - 1)]
        elif fam == "complete":
            e = [(i, j, W) for i in range(n) for j in range(i + 1, n)]
        elif fam == "mesh":
            R, C = g["rows"], g["cols"]
            e = [(r * C + c, r * C + c + 1, W) for r in range(R) for c in range(C - 1)]
            e += [(r * C + c, (r + 1) * C + c, W) for r in range(R - 1) for c in range(C)]
        a = np.array(e, np.uint32).reshape(-1, 3)
        out.append((g["name"], n, a[:, 0].copy(), a[:, 1].copy(), a[:, 2].copy(), g["diameter"]))
    return out
