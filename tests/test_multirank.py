"""Multi-rank frame sharding on CPU ranks (gloo, world size 2): disjoint frame
sets, per-rank results independent of the other rank, max-over-ranks timing."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import oracle
    import synth
    from paper_2411_01919_b300.shard import max_over_ranks, rank_frame_seeds
    dist.init_process_group('gloo', init_method='tcp://127.0.0.1:%d' % port, rank=rank,
                            world_size=world)
    seeds = rank_frame_seeds(rank, world, 2)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    planes = []
    for s in seeds:
        fr = synth.frame_c1(s)
        r = oracle.process_frame(fr.encoded, fr.dtype, fr.cam.intrinsics, 3, hypotheses=64,
                                 max_planes=2, min_inliers=100, seed=1, frame_idx=s)
        planes.append(r.ransac.planes.tolist())
    m = max_over_ranks(float(rank + 1))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, gathered, planes, m))


def test_two_cpu_ranks_shard_frames_without_exchanging_them():
    ctx = mp.get_context('spawn')
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        rank, gathered, planes, m = q.get(timeout=240)
        res[rank] = (gathered, planes, m)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g0 = res[0][0]
    assert set(g0[0]).isdisjoint(g0[1])
    assert res[0][2] == res[1][2] == 2.0
    # a rank's result depends only on its own frames: recompute rank 1 alone
    import oracle
    import synth
    for s, pl in zip(g0[1], res[1][1]):
        fr = synth.frame_c1(s)
        r = oracle.process_frame(fr.encoded, fr.dtype, fr.cam.intrinsics, 3, hypotheses=64,
                                 max_planes=2, min_inliers=100, seed=1, frame_idx=s)
        assert np.array_equal(np.array(pl).reshape(-1, 4), r.ransac.planes)


def test_rank_seeds_reject_bad_ranks():
    from paper_2411_01919_b300.shard import rank_frame_seeds
    with pytest.raises(ValueError):
        rank_frame_seeds(2, 2, 4)
    assert rank_frame_seeds(1, 4, 3) == [1000, 1001, 1002]
