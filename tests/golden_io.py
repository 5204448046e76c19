"""Loader for the hand-enumerated fixtures in tests/golden/ (shared by the
oracle pins and the GPU parity tests)."""
import glob
import json
import math
import os

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
P_OF = {"1": 1.0, "2": 2.0, "inf": math.inf, "-inf": -math.inf, "-1": -1.0, "3": 3.0}


def closed_form(expr: str) -> float:
    """Evaluates the closed forms used in the fixtures: "a/b", "sqrt(a/b)",
    "cbrt(a/b)", "a"."""
    expr = expr.strip()
    if expr.startswith("sqrt(") and expr.endswith(")"):
        return math.sqrt(closed_form(expr[5:-1]))
    if expr.startswith("cbrt(") and expr.endswith(")"):
        return closed_form(expr[5:-1]) ** (1.0 / 3.0)
    if "/" in expr:
        a, b = expr.split("/")
        return float(int(a)) / float(int(b))
    return float(int(expr))


def load_all():
    out = []
    for path in sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.json"))):
        with open(path) as f:
            d = json.load(f)
        e = np.array(d["edges"], dtype=np.int64).reshape(-1, 3)
        d["u"] = e[:, 0].astype(np.int32)
        d["v"] = e[:, 1].astype(np.int32)
        d["w"] = e[:, 2].astype(np.int32)
        d["name"] = os.path.basename(path)
        out.append(d)
    return out
