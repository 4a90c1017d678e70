"""Host logic of the partitioned right-hand side (Sec. 3.6 int/mpi split), on
CPU with host-only contexts: every pair is either interior to one partition
or shared by exactly two with the same exchange slots on both sides, and
ranks built in separate processes (gloo, world size 2) agree on the slots."""

import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from fr_inputs import periodic_box, annulus_mixed
from tests.libutil import ensure_built


@pytest.fixture(scope="module")
def fr():
    ensure_built()
    from paper_1312_1638_b300 import fr as _fr
    return _fr


def _mixed():
    return annulus_mixed(ntheta=12, nr_quad=2, nr_tri=2, r0=0.5, r1=3.0, jitter=0.05, seed=1)


def _partition(mesh, nparts, seed):
    """Random partition with every block present in every part."""
    rng = np.random.default_rng(seed)
    parts = []
    for b in mesh.blocks:
        p = rng.integers(0, nparts, b.nodes.shape[0])
        p[:nparts] = np.arange(nparts)
        parts.append(p)
    return np.concatenate(parts).astype(np.int32)


def _global_side(mesh, part):
    base = np.cumsum([0] + [b.nodes.shape[0] for b in mesh.blocks])
    return lambda blk, e: part[base[blk] + e]


@pytest.mark.parametrize("case,nparts", [("hex", 2), ("hex", 3), ("mixed", 2), ("mixed", 4)])
def test_pairs_split_into_interior_and_shared(fr, case, nparts):
    mesh = periodic_box("hex", 3, 0.0, 1.0, jitter=0.1, seed=1) if case == "hex" else _mixed()
    part = _partition(mesh, nparts, seed=nparts)
    whole = fr.Solver(mesh, 2, "euler", "fp64", device=-1)
    gp = whole.pairs()                                   # (bL, fL, nL, bR, fR, nR)
    side = _global_side(mesh, part)
    pl = np.array([side(r[0], r[2]) for r in gp])
    pr = np.array([side(r[3], r[5]) for r in gp])
    ranks = [fr.Solver(mesh, 2, "euler", "fp64", device=-1, part=part, nparts=nparts, rank=r) for r in range(nparts)]
    # interior pairs: one per global pair with both sides on the same rank
    assert sum(len(s.pairs()) for s in ranks) == int(np.sum(pl == pr))
    slots = [s.part_slots() for s in ranks]
    for p in range(nparts):
        for q, keys in slots[p].items():
            assert q != p
            assert np.array_equal(keys, slots[q][p])     # both sides list the same slots in the same order
            # the slots are exactly the global pairs between p and q, keyed by the global L side
            want = {tuple(r[[0, 2, 1]]) for r, a, b in zip(gp, pl, pr) if {a, b} == {p, q}}
            assert {tuple(k) for k in keys} == want and len(keys) == len(want)
            # pairs whose L side lies on the lower rank come first, each part sorted
            lower = min(p, q)
            first = np.array([side(k[0], k[1]) == lower for k in keys])
            nf = int(first.sum())
            assert first[:nf].all() and not first[nf:].any()
            for seg in (keys[:nf], keys[nf:]):
                assert all(tuple(a) < tuple(b) for a, b in zip(seg[:-1], seg[1:]))
    # every cross pair is counted once on each side
    assert sum(len(k) for sl in slots for k in sl.values()) == 2 * int(np.sum(pl != pr))


def test_partition_must_keep_every_block(fr):
    mesh = _mixed()
    part = np.zeros(sum(b.nodes.shape[0] for b in mesh.blocks), np.int32)
    part[:5] = 1                                         # rank 1 gets quads only
    with pytest.raises(fr.FRError) as e:
        fr.Solver(mesh, 2, "euler", "fp64", device=-1, part=part, nparts=2, rank=1)
    assert e.value.status == fr.ERR_ARG
    with pytest.raises(fr.FRError):
        fr.Solver(mesh, 2, "euler", "fp64", device=-1, part=part, nparts=2, rank=2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1312_1638_b300 import fr as _fr
    mesh = periodic_box("quad", 6, 0.0, 1.0, jitter=0.1, seed=2)
    part = (np.arange(36) % 6 >= 3).astype(np.int32)      # left / right halves
    s = _fr.Solver(mesh, 3, "ns", "fp64", device=-1, part=part, nparts=world, rank=rank)
    mine = {q: k.tolist() for q, k in s.part_slots().items()}
    allk = [None] * world
    dist.all_gather_object(allk, mine)
    ok = all(allk[q][p] == allk[p][q] for p in range(world) for q in allk[p])
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{int(ok)} {sum(len(v) for v in mine.values())}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_agree_on_exchange_slots(fr, tmp_path):
    mp.start_processes(_rank_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    res = [open(tmp_path / f"r{r}.txt").read().split() for r in range(2)]
    assert all(r[0] == "1" for r in res)
    # a 6x6 periodic box cut in two halves shares two 6-cell columns of faces, 4 flux points each (p = 3)
    assert int(res[0][1]) == int(res[1][1]) == 2 * 6 * 4
