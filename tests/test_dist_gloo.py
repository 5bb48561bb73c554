"""Multi-process host logic of the sharded path (paper_2309_03308_gb300.dist)
on CPU: two gloo ranks shard an all-pairs region pair by rows and a list of
region pairs, compute their shares with the FP64 oracle, and exchange only
the extremes; the merged result equals the unsharded oracle result."""
import os
import socket

import numpy as np
import pytest

import gen
import oracle
from gen import configs
from paper_2309_03308_gb300 import dist as D

X, Y, Z, N = 16, 16, 4, 32
BOX_A = (0, 0, 0, 8, 8, 4)
BOX_B = (8, 8, 0, 16, 16, 4)


def field_with_cross_shard_tie():
    F = gen.field(configs.SMALL["seed"], X, Y, Z, N).reshape(N, -1).copy()
    q = 8 + 16 * (8 + 16 * 0)  # a point of B
    # two points of A in different z-slabs get q's vector: r = 1 at both pairs
    for p in (3 + 16 * (2 + 16 * 0), 5 + 16 * (1 + 16 * 3)):
        F[:, p] = F[:, q]
    return F.reshape(N, Z, Y, X)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, F):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        orc = oracle.get()
        orc.set_threads(1)
        B = oracle.box_points(X, Y, Z, BOX_B)
        # (1) rows of one region pair, both extremes, for Pearson and KSG
        for kind in (oracle.PEARSON, oracle.MI_KSG):
            (sub, first), = [s for i, s in enumerate(D.split_box(BOX_A, world)) if i == rank]
            res = orc.region_extremes(F, oracle.box_points(X, Y, Z, sub), B, False, kind, k=3)
            for key in ("argmax", "argmin"):
                res[key] = D.shift_pair_index(res[key], first, len(B))
            (merged,) = D.allreduce_extremes([res])
            full = orc.region_extremes(F, oracle.box_points(X, Y, Z, BOX_A), B, False, kind, k=3)
            assert merged == full, (kind, merged, full)
        # (2) a list of region pairs, contiguous shares, gathered
        boxes = configs.regular_boxes(X, Y, Z, 8, 8, 2)
        rps = [(i, j) for i in range(len(boxes)) for j in range(i, len(boxes))]
        lo, hi = D.shard_range(len(rps), rank, world)
        mine = [orc.region_extremes(F, oracle.box_points(X, Y, Z, boxes[i]),
                                    oracle.box_points(X, Y, Z, boxes[j]), i == j,
                                    oracle.SPEARMAN) for i, j in rps[lo:hi]]
        allr = D.allgather_shards(mine)
        if rank == 0:
            ref = [orc.region_extremes(F, oracle.box_points(X, Y, Z, boxes[i]),
                                       oracle.box_points(X, Y, Z, boxes[j]), i == j,
                                       oracle.SPEARMAN) for i, j in rps]
            assert allr == ref
    finally:
        dist.destroy_process_group()


def test_shard_range_covers_once():
    for n in (0, 1, 7, 36, 3916):
        for world in (1, 2, 3, 8):
            parts = [D.shard_range(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            sizes = [hi - lo for lo, hi in parts]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("box", [(0, 0, 0, 8, 8, 4), (2, 3, 1, 9, 7, 2), (1, 1, 0, 9, 2, 1)])
def test_split_box_is_contiguous_in_enumeration(box):
    full = oracle.box_points(X, Y, Z, box)
    for parts in (1, 2, 3, 5):
        got = []
        for sub, first in D.split_box(box, parts):
            pts = oracle.box_points(X, Y, Z, sub)
            assert np.array_equal(full[first:first + len(pts)], pts)
            got.append(pts)
        assert np.array_equal(np.concatenate(got), full)


def test_merge_tie_goes_to_smaller_index():
    a = dict(max=1.0, min=-0.5, argmax=40, argmin=7, count=10)
    b = dict(max=1.0, min=-0.5, argmax=12, argmin=9, count=5)
    m = D.merge_extremes([a, b])
    assert m == dict(max=1.0, min=-0.5, argmax=12, argmin=7, count=15)
    assert D.merge_extremes([a, dict(D._EMPTY)]) == a


def test_two_gloo_ranks_match_unsharded_oracle():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    oracle.get()  # build the oracle library once, before the ranks start
    F = field_with_cross_shard_tie()
    mp.spawn(_worker, args=(2, _free_port(), F), nprocs=2, join=True)
    del torch
