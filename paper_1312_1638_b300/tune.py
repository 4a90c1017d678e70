"""Autotune the tensor-core kernel variants for the standard workloads and
write the table that fr.Solver.apply_tuning() reads.

usage: python -m paper_1312_1638_b300.tune [OUT.json] [--only KEY ...]

Each workload's solver runs fr_autotune on its own synthetic state (the
benchmark's Taylor-Green states, the mixed annulus' free stream plus a
seeded perturbation); the chosen variants are stored under the solver's
tuning key (element types / order / system / precision).  Needs a GPU.
"""

from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

TG = dict(gamma=1.4, mu=1.0 / 1600.0, prandtl=0.71, ldg_beta=0.5, ldg_tau=0.1, ref_rho=1.0,
          ref_p=1.0 / (1.4 * 0.1 ** 2))


def _workloads():
    """(name, mesh factory, order, system, precision, params, state factory)."""
    from fr_inputs import periodic_box, annulus_mixed, fields
    p_inf = 1.0 / (1.4 * 0.2 ** 2)
    mixed = dict(gamma=1.4, mu=0.01, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1, bc_rho=1.0, bc_v=(1.0, 0.0, 0.0),
                 bc_p=p_inf, outflow_p=p_inf, wall_cpTw=1.4 / 0.4 * p_inf, ref_rho=1.0, ref_p=p_inf)
    tg = lambda X: fields.perturbed_taylor_green(X, M=0.1)
    out = []
    for prec in ("tf32x3", "bf16x3"):
        out.append((f"hex96_p4_ns_{prec}", lambda: periodic_box("hex", 96, 0.0, 2 * np.pi), 4, "ns", prec, TG, tg))
        out.append((f"hex32_p3_ns_{prec}", lambda: periodic_box("hex", 32, 0.0, 2 * np.pi), 3, "ns", prec, TG, tg))
        out.append((f"annulus_p4_ns_{prec}", annulus_mixed, 4, "ns", prec, mixed,
                    lambda X: fields.smooth_random(X, seed=3, amp=0.1, vel0=(1.0, 0.0), p0=p_inf)))
        out.append((f"hex16_p4_euler_{prec}", lambda: periodic_box("hex", 16, 0.0, 2 * np.pi), 4, "euler", prec,
                    dict(gamma=1.4, ref_rho=1.0, ref_p=TG["ref_p"]), tg))
    return out


def main(argv):
    import torch
    from paper_1312_1638_b300 import fr
    out = argv[0] if argv and not argv[0].startswith("--") else fr.TUNING_CACHE
    only = argv[argv.index("--only") + 1:] if "--only" in argv else None
    table = json.load(open(out)) if os.path.exists(out) else {}
    for name, mk, order, system, prec, prm, st in _workloads():
        if only and name not in only:
            continue
        m = mk()
        s = fr.Solver(m, order, system, prec, device=0, **prm)
        u = []
        for b in range(len(m.blocks)):
            X = s.solution_points(b)
            u.append(torch.from_numpy(s.pack(b, np.asarray(st(X)).transpose(1, 0, 2))).cuda())
        text = s.autotune(u, reps=2)
        table[s.tuning_key()] = text
        print(f"{name:24s} {s.tuning_key():32s} {text}", flush=True)
        s.close()
        del u
        torch.cuda.empty_cache()
    with open(out, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:])
