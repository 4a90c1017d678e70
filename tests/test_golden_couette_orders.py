"""The order-of-accuracy fit used by the Couette study (least-squares slope of
log sigma against log h, with its standard error) reproduces the orders the
paper prints from its own errors (Sec. 5.2; tests/golden/couette_sigma_tables.txt,
2D mixed meshes with h ~ N_E^-1/2 for N_E = triangles + quadrilaterals, 3D
extruded and unstructured hexahedra).  The printed errors carry three
significant digits, so orders and standard errors agree to 0.015."""

import os

import numpy as np
import pytest

from tests.couette_study import order

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "couette_sigma_tables.txt")


def _tables():
    tabs, cur = [], None
    for line in open(GOLDEN):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "table":
            cur = dict(name=line[1], expo=float(line[2]), rows=[], order=None)
            tabs.append(cur)
        elif line[0] == "order":
            cur["order"] = [float(x) for x in line[1:]]
        else:
            cur["rows"].append([float(x) for x in line])
    return tabs


@pytest.mark.parametrize("tab", _tables(), ids=lambda t: t["name"])
def test_order_fit_reproduces_printed_orders(tab):
    rows = np.array(tab["rows"])
    h = rows[:, 0] ** tab["expo"]
    printed = np.array(tab["order"]).reshape(-1, 2)
    assert len(printed) == rows.shape[1] - 1
    for p, (o_ref, se_ref) in enumerate(printed, start=1):
        o, se = order(h, rows[:, p])
        assert abs(o - o_ref) <= 0.015, (tab["name"], p, o, o_ref)
        assert abs(se - se_ref) <= 0.015, (tab["name"], p, se, se_ref)
