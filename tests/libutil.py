"""Shared helpers for the library tests: build-once fixture and comparison
with the oracle."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def ensure_built():
    from paper_1312_1638_b300 import build
    return build.build()


def declared_functions():
    """Function names declared in include/*.h."""
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            src = open(os.path.join(inc, fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(fr_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def oracle_state(osys, fn):
    return [fn(osys.solution_coords(b)).transpose(1, 0, 2).copy() for b in range(len(osys.eles))]


def rel_l2_per_var(x, ref):
    """max over variables of ||x - ref||_2 / ||ref||_2 (arrays [npts, nvars, nelem])."""
    num = np.sqrt(((x - ref) ** 2).sum(axis=(0, 2)))
    den = np.sqrt((ref ** 2).sum(axis=(0, 2)))
    return float((num / np.maximum(den, 1e-300)).max())
