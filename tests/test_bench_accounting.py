"""The roofline accounting of bench.py (CPU): the algorithmic bytes and
operator flops it divides by kernel time, against the per-unit figures for
the benchmark workload (hex p=4, Navier-Stokes, FP32 values): 2.44 MFLOP of
operator products per element (3,900 flop per DOF, 2.16 TFLOP per RHS on the
96^3 box), every value moved once per kernel."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

NU, NF, V, D, S = 125, 150, 5, 3, 4          # hex p=4: (p+1)^3 solution, 6 (p+1)^2 flux points
E96 = 96 ** 3


def test_operator_flops_per_element_and_per_rhs():
    per_elem = bench.operator_flops_per_rhs(NU, NF, V, D, 1)
    assert per_elem == pytest.approx(2.4375e6)                    # 2.44 MFLOP / element
    assert per_elem / (NU * V) == pytest.approx(3900.0)           # flop / DOF
    assert bench.operator_flops_per_rhs(NU, NF, V, D, E96) == pytest.approx(2.157e12, rel=1e-3)


@pytest.mark.parametrize("name,fused,bytes_per_elem,flops_per_elem", [
    ("disu_gemm", False, (125 + 150) * 5 * 4, 2 * 150 * 125 * 5),
    ("gradfpts_gemm", False, (125 + 150) * 5 * 4, 2 * 150 * 125 * 5),
    # C (150), U (125) in, Q (3 x 125) out, per variable; adj(J) (9) and 1/J per point
    ("tgradu_gemm", True, ((150 + 125 + 375) * 5 + 10 * 125) * 4, 2 * 375 * 275 * 5),
    ("tgradu_gemm", False, (150 + 125 + 375) * 5 * 4, 2 * 375 * 275 * 5),
    # D~ (150) and F~ (375) in per variable, 1/J per point; fused RK stage: 3, 4, 4, 2 values per entry
    ("tdivf_gemm", True, ((150 + 375) * 5 + 125) * 4 + 13 * 125 * 5 * 4 / 4, 2 * 125 * 525 * 5),
    ("tdivf_gemm", False, ((150 + 375 + 125) * 5 + 125) * 4, 2 * 125 * 525 * 5),
    # U (5) and Q (15) in, F~ (15) out, adj(J) (9) per point
    ("tdisf", False, (5 + 15 + 15 + 9) * 125 * 4, 0),
    ("gradcoru", False, (2 * 15 + 9 + 1) * 125 * 4, 0),
])
def test_kernel_work_per_element(name, fused, bytes_per_elem, flops_per_elem):
    b, f = bench.kernel_work(name, NU, NF, V, D, 1, 0, S, fused=fused)
    assert b == pytest.approx(bytes_per_elem)
    assert f == pytest.approx(flops_per_elem)


def test_interface_kernel_work_per_pair():
    # both sides' U^(f) read and written (comm_sol writes C to both sides); two
    # uint32 offsets per pair
    assert bench.kernel_work("comm_sol", NU, NF, V, D, 0, 1, S)[0] == 4 * 5 * 4 + 8
    # + both sides' Q^(f), the normal (3) and J^(f) n^(f) of both sides
    assert bench.kernel_work("comm_flux", NU, NF, V, D, 0, 1, S)[0] == (4 * 5 + 2 * 3 * 5 + 3 + 2) * 4 + 8
    # LDG beta = +-1/2: the zero-weight side's U^(f) (common solution) and Q^(f)
    # (viscous common flux) are not read
    assert bench.kernel_work("comm_sol", NU, NF, V, D, 0, 1, S, one_side=True)[0] == 3 * 5 * 4 + 8
    assert bench.kernel_work("comm_flux", NU, NF, V, D, 0, 1, S, one_side=True)[0] == (4 * 5 + 3 * 5 + 3 + 2) * 4 + 8


def test_dominant_kernel_bytes_at_full_size():
    # the roofline line's algorithmic bytes for the fused gradient GEMM on the 96^3 box
    b, f = bench.kernel_work("tgradu_gemm", NU, NF, V, D, E96, 0, S, fused=True)
    assert b == 15925248000
    assert f == pytest.approx(912384000000.0)
