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


def kappa_per_var(S, R):
    """Condition of each variable's RHS: ||S_v||_2 / ||R_v||_2 (arrays [npts, nvars, nelem])."""
    num = np.sqrt((S ** 2).sum(axis=(0, 2)))
    den = np.sqrt((R ** 2).sum(axis=(0, 2)))
    return num / np.maximum(den, 1e-300)


def rel_l2_vars(x, ref):
    """||x_v - ref_v||_2 / ||ref_v||_2 for every variable v (arrays [npts, nvars, nelem])."""
    num = np.sqrt(((x - ref) ** 2).sum(axis=(0, 2)))
    den = np.sqrt((ref ** 2).sum(axis=(0, 2)))
    return num / np.maximum(den, 1e-300)


def record_parity(case, prec, **fields):
    """Append one JSON line of measured errors to the file named by
    FR_PARITY_LOG (nothing when it is unset)."""
    import json
    path = os.environ.get("FR_PARITY_LOG")
    if not path:
        return
    rec = dict(case=case, precision=prec)
    for k, v in fields.items():
        rec[k] = [float(x) for x in v] if hasattr(v, "__len__") else float(v)
    with open(path, "a") as fh:
        fh.write(json.dumps(rec) + "\n")


def m0_spread(osys, U, samples=2, ulps=8, seed=7):
    """Per block, per variable: the largest change of the oracle's RHS when the
    entries of every element type's interpolation operator M0 are perturbed by
    up to `ulps` units in the last place (seeded samples).  FP64 results of two
    exact-equivalent constructions of M0 differ at that level, and the RHS
    amplifies it (Sec. 2 operators evaluated in FP64); computed from the
    oracle alone."""
    R0 = osys.rhs(U)
    saved = [el.M0.copy() for el in osys.eles]
    rng = np.random.default_rng(seed)
    spread = [np.zeros(r.shape[1]) for r in R0]
    try:
        for _ in range(samples):
            for el, M0 in zip(osys.eles, saved):
                el.M0 = M0 * (1 + ulps * np.finfo(float).eps * rng.uniform(-1, 1, M0.shape))
            for b, r in enumerate(osys.rhs(U)):
                spread[b] = np.maximum(spread[b], np.abs(r - R0[b]).max(axis=(0, 2)))
    finally:
        for el, M0 in zip(osys.eles, saved):
            el.M0 = M0
    return spread
