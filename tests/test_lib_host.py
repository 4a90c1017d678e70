"""CPU tests of the C-ABI library: it loads, exports every function declared
in include/fr.h, and its host-side set-up (operators, solution points,
interface pairs, error statuses) agrees with the oracle.  No compute calls
are made (no GPU here)."""
import ctypes
import os

import numpy as np
import pytest

from tests.libutil import ensure_built, declared_functions
from fr_inputs import periodic_box, annulus_mixed, Mesh, Block
from oracle.system import FRSystem


@pytest.fixture(scope="module")
def fr():
    ensure_built()
    from paper_1312_1638_b300 import fr as frmod
    return frmod


def test_library_exports_every_declared_symbol(fr):
    lib = ctypes.CDLL(fr.LIBPATH)
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(fr.EXPORTS)
    assert fr.load().fr_version() == 6


CASES = [("quad", 3, 1, 0.1), ("quad", 3, 4, 0.1), ("hex", 2, 2, 0.1), ("hex", 2, 4, 0.0)]


@pytest.mark.parametrize("etype,n,p,jit", CASES)
def test_operators_and_points_match_oracle(fr, etype, n, p, jit):
    m = periodic_box(etype, n, 0.0, 2 * np.pi, jitter=jit, seed=1)
    s = fr.Solver(m, p, "ns", "fp64", device=-1)
    o = FRSystem(m, p, "ns")
    el = o.eles[0]
    for which, M in [(0, el.M0), (1, el.M1), (2, el.M2), (3, el.M3), (4, el.M4), (6, el.M6),
                     (7, el.M4 - el.M6 @ el.M0), (8, el.M1 - el.M3 @ el.M2)]:
        assert np.allclose(s.operator(0, which), M, atol=1e-12), which
    assert np.allclose(s.solution_points(0), o.solution_coords(0), atol=1e-13)


@pytest.mark.parametrize("corr", ["sd", "hu"])
@pytest.mark.parametrize("etype,p", [("quad", 1), ("quad", 4), ("hex", 2), ("hex", 3)])
def test_vcjh_operators_match_oracle(fr, etype, p, corr):
    m = periodic_box(etype, 2, 0.0, 1.0, jitter=0.1, seed=1)
    s = fr.Solver(m, p, "ns", "fp64", device=-1, correction=corr)
    el = FRSystem(m, p, "ns", correction=corr).eles[0]
    for which, M in [(3, el.M3), (6, el.M6), (7, el.M4 - el.M6 @ el.M0), (8, el.M1 - el.M3 @ el.M2)]:
        assert np.allclose(s.operator(0, which), M, atol=1e-12), which
    assert not np.allclose(s.operator(0, 3), FRSystem(m, p, "ns").eles[0].M3)


def test_vcjh_on_triangles_is_unsupported(fr):
    from fr_inputs import annulus_mixed
    m = annulus_mixed(ntheta=12, nr_quad=2, nr_tri=2, r0=0.5, r1=3.0, jitter=0.0, seed=1)
    with pytest.raises(fr.FRError) as e:
        fr.Solver(m, 2, "euler", "fp64", device=-1, correction="sd")
    assert e.value.status == fr.ERR_UNSUPPORTED


def _pair_set(rows):
    return {tuple(int(v) for v in r) for r in rows}


@pytest.mark.parametrize("etype,n,p,jit", CASES[:3])
def test_pairs_match_oracle(fr, etype, n, p, jit):
    m = periodic_box(etype, n, 0.0, 1.0, jitter=jit, seed=4, shuffle=True)
    s = fr.Solver(m, p, "euler", "fp64", device=-1)
    o = FRSystem(m, p)
    P = o.pairs
    ref = np.stack([P["bL"], P["fL"], P["nL"], P["bR"], P["fR"], P["nR"]], 1)
    assert _pair_set(s.pairs()) == _pair_set(ref)


def test_mixed_mesh_setup_matches_oracle(fr):
    m = annulus_mixed(ntheta=16, nr_quad=2, nr_tri=2, r0=0.5, r1=3.0, jitter=0.05, seed=3)
    s = fr.Solver(m, 3, "ns", "fp64", device=-1)
    o = FRSystem(m, 3, "ns")
    for b in range(2):
        el = o.eles[b]
        for which, M in [(0, el.M0), (3, el.M3), (4, el.M4)]:
            assert np.allclose(s.operator(b, which), M, atol=1e-12)
        assert np.allclose(s.solution_points(b), o.solution_coords(b), atol=1e-13)
    P = o.pairs
    ref = np.stack([P["bL"], P["fL"], P["nL"], P["bR"], P["fR"], P["nR"]], 1)
    assert _pair_set(s.pairs()) == _pair_set(ref)


def test_layout_padding(fr):
    m = periodic_box("hex", 3, jitter=0.0)
    s = fr.Solver(m, 2, "euler", "fp32", device=-1)
    L = s.layout(0)
    assert L == dict(nupts=27, nfpts=54, nvars=5, nelem=27, ld=128)


def test_unmatched_face_is_a_mesh_error(fr):
    m = periodic_box("quad", 3)
    m.periodic = m.periodic[:1]           # drop the y identification
    with pytest.raises(fr.FRError) as e:
        fr.Solver(m, 2, device=-1)
    assert e.value.status == fr.ERR_MESH


def test_inverted_element_is_a_mesh_error(fr):
    m = periodic_box("quad", 2)
    nodes = m.blocks[0].nodes.copy()
    nodes[0] = nodes[0][[1, 0, 3, 2]]     # mirror one element
    m2 = Mesh(2, [Block("quad", nodes)], m.bfaces, m.periodic)
    with pytest.raises(fr.FRError) as e:
        fr.Solver(m2, 2, device=-1)
    assert e.value.status == fr.ERR_MESH


def test_bad_arguments(fr):
    m = periodic_box("quad", 2)
    with pytest.raises(fr.FRError) as e:
        fr.Solver(m, 0, device=-1)
    assert e.value.status == fr.ERR_ARG
    s = fr.Solver(m, 1, device=-1)
    assert s.lib.fr_rhs(s.ctx, None, None, None) in (fr.ERR_ARG, fr.ERR_UNSUPPORTED)
    assert s.lib.fr_layout(s.ctx, 5, None, None, None, None, None) == fr.ERR_ARG


def test_context_options_are_validated(fr):
    m = periodic_box("quad", 2, 0.0, 1.0)
    s = fr.Solver(m, 1, "euler", "tf32x3", device=-1)
    s.set_option("graphs", 0)
    s.set_option("tc_wait_limit", 1000)
    s.set_option("tc_wait_limit", 0)                     # back to the default limit
    with pytest.raises(fr.FRError) as e:
        s.set_option("tc_wait_limit", -1)
    assert e.value.status == fr.ERR_ARG
    with pytest.raises(fr.FRError) as e:
        s.set_option("no_such_option", 1)
    assert e.value.status == fr.ERR_ARG


def test_every_abi_declaration_cites_its_passage():
    """Each entry point of include/fr.h is preceded by a comment that cites the
    paper passage defining it (Sec., Eq., App.) or says it is not in the paper."""
    import re
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fr.h")).read()
    decls = list(re.finditer(r"^(?:fr_status|int32_t|const char\*|void)\s+(fr_\w+)\(", src, re.M))
    assert len(decls) >= 20
    bad = []
    for m in decls:
        # skip #defines and the declarations of a group that shares one comment
        lines = src[:m.start()].rstrip().split("\n")
        while lines and (not lines[-1].strip() or lines[-1].startswith("#define")
                         or re.match(r"^(fr_status|int32_t|const char\*|void)\s+fr_\w+\(", lines[-1])
                         or (lines[-1].startswith("    ") and lines[-1].rstrip().endswith(");"))):
            lines.pop()
        before = "\n".join(lines)
        if not before.rstrip().endswith("*/"):
            bad.append((m.group(1), "no comment"))
            continue
        c = before[before.rfind("/*"):]
        if not re.search(r"Sec\.|Eq\.|App\.|not in the paper", c):
            bad.append((m.group(1), "no citation"))
    assert not bad, bad


@pytest.mark.parametrize("entry", [(1, 0, 0, 2), (0, 99, 0, 2), (0, 0, 7, 2), (0, 0, 0, 4), (0, 0, 0, -1)])
def test_bad_boundary_entry_is_a_mesh_error(fr, entry):
    # an unknown block, element, face or boundary type in the boundary list
    m = periodic_box("quad", 3)
    m.periodic = m.periodic[:1]                          # y faces become boundaries
    import numpy as np
    ny = [(0, e, f, 2) for e in range(9) for f in range(4) if (f == 0 and e < 3) or (f == 2 and e >= 6)]
    fr.Solver(Mesh(2, m.blocks, np.array(ny, dtype=np.int64), m.periodic), 1, device=-1)   # the valid list
    bf = np.array(ny + [entry], dtype=np.int64)
    m2 = Mesh(2, m.blocks, bf, m.periodic)
    with pytest.raises(fr.FRError) as e:
        fr.Solver(m2, 1, device=-1)
    assert e.value.status in (fr.ERR_MESH, fr.ERR_ARG)


def test_paired_face_listed_as_boundary_is_a_mesh_error(fr):
    import numpy as np
    m = periodic_box("quad", 3)
    m2 = Mesh(2, m.blocks, np.array([(0, 4, 1, 2)], dtype=np.int64), m.periodic)   # an interior face
    with pytest.raises(fr.FRError) as e:
        fr.Solver(m2, 1, device=-1)
    assert e.value.status == fr.ERR_MESH


def test_device_calls_on_a_host_only_context_are_refused(fr):
    m = periodic_box("quad", 2)
    s = fr.Solver(m, 1, "ns", "fp64", device=-1, mu=0.01)
    assert s.lib.fr_adjoint_rhs(s.ctx, None, None, None, None) in (fr.ERR_ARG, fr.ERR_UNSUPPORTED)
    assert s.lib.fr_rk4(s.ctx, None, 1e-3, 1, None) in (fr.ERR_ARG, fr.ERR_UNSUPPORTED)
    assert s.lib.fr_sync_status(s.ctx) == fr.ERR_UNSUPPORTED


def test_tuning_calls_on_host_only_contexts(fr):
    """fr_get_tuning reports no blocks on a host-only context, fr_set_tuning
    refuses (it chooses device kernels)."""
    m = periodic_box("hex", 2, 0.0, 1.0)
    s = fr.Solver(m, 2, "ns", "tf32x3", device=-1)
    assert s.tuning() == ""
    with pytest.raises(fr.FRError) as e:
        s.set_tuning("b0:disu=1.8.3")
    assert e.value.status == fr.ERR_UNSUPPORTED
    assert "tf32x3" in s.tuning_key() and s.tuning_key().startswith("hex/p2/ns")
