"""Served and batched forms on the GPU: continuous batching returns for every
request exactly what the frame gives alone; admission respects the memory
budget; the autotuner leaves results unchanged."""
import numpy as np
import pytest
import torch

import synth
from paper_2411_01919_b300 import Params, Pipeline
from paper_2411_01919_b300.serve import Request, Server, poisson_arrivals, summarize
from paper_2411_01919_b300.tune import DiffusionTuner

pytestmark = pytest.mark.gpu

P = Params(iters=12, hypotheses=256, max_planes=5, min_inliers=100, seed=4)


def pool(n_streams=4, poses=2):
    fr = synth.stream_pool(n_streams, poses, seed=3, workers=0)
    host = {s: [torch.from_numpy(np.ascontiguousarray(f.encoded)).pin_memory() for f in v]
            for s, v in fr.items()}
    return fr, host


def alone(frames_by_stream, reqs):
    """Every request processed alone through pm_process_frame."""
    out = {}
    mw = max(f.w for v in frames_by_stream.values() for f in v)
    mh = max(f.h for v in frames_by_stream.values() for f in v)
    with Pipeline(P, mw, mh, 1) as pipe:
        for r in reqs:
            d = r.depth.cuda()
            out[(r.stream, r.k)] = pipe.process_frame(d, r.K, frame_idx=r.frame_idx, labels=False)
    return out


def make_reqs(fr, host, arrivals, poses):
    return [Request(s, k, t, host[s][k % poses], fr[s][k % poses].cam.intrinsics, frame_idx=k)
            for s, k, t in arrivals]


def test_served_results_equal_alone_under_realtime_load():
    fr, host = pool()
    arr = poisson_arrivals(4, 1.5, 1 / 30, seed=5)
    reqs = make_reqs(fr, host, arr, 2)
    srv = Server(P, budget_bytes=4 << 30, max_batch=8, n_lanes=2)
    out = srv.run(reqs, realtime=True)
    st = summarize(out, srv.elapsed)
    srv.close()
    assert st['refused'] == 0 and st['frames'] == len(reqs)
    assert srv.stats['batches'] >= 2
    ref = alone(fr, out)
    for r in out:
        a, b = r.planes, ref[(r.stream, r.k)]
        assert np.array_equal(a.planes, b.planes) and np.array_equal(a.n_inliers, b.n_inliers)


def test_saturated_mix_batches_and_matches_alone():
    fr, host = pool()
    reqs = make_reqs(fr, host, [(s, k, 0.0) for k in range(6) for s in range(4)], 2)
    srv = Server(P, budget_bytes=4 << 30, max_batch=8, n_lanes=2)
    out = srv.run(reqs, realtime=False)
    srv.close()
    assert srv.stats['batched_frames'] == len(reqs)
    assert srv.stats['batches'] < len(reqs)          # frames really shared launches
    ref = alone(fr, out)
    for r in out:
        assert np.array_equal(r.planes.planes, ref[(r.stream, r.k)].planes)


def test_full_batches_replay_graphs_and_match_alone():
    """Under saturation every batch is full, so the lanes replay CUDA graphs
    (captured once per lane and batch shape); results equal each frame alone."""
    fr, host = pool(8, 2)
    reqs = make_reqs(fr, host, [(s, k, 0.0) for k in range(4) for s in range(8)], 2)
    srv = Server(P, budget_bytes=8 << 30, max_batch=4, n_lanes=2)
    out = srv.run(reqs, realtime=False)
    srv.close()
    assert srv.stats['graph_batches'] == srv.stats['batches'] == len(reqs) // 4
    ref = alone(fr, out)
    for r in out:
        a, b = r.planes, ref[(r.stream, r.k)]
        assert np.array_equal(a.planes, b.planes) and np.array_equal(a.n_inliers, b.n_inliers)


def test_malformed_requests_are_refused_alone():
    """Requests that cannot be served -- bad intrinsics, a frame larger than
    the lanes, a stream that changes its frame size -- are refused with a
    reason at admission; every other request is served as it is alone."""
    fr, host = pool()
    reqs = make_reqs(fr, host, [(s, k, 0.0) for k in range(4) for s in range(4)], 2)
    big = torch.zeros((8, 4000), dtype=torch.float32).pin_memory()
    odd = torch.zeros((7, 9), dtype=torch.float32).pin_memory()
    bad = [Request(0, 100, 0.0, host[0][0], (0.0, 0.0, 1.0, 1.0), frame_idx=100),
           Request(9, 0, 0.0, big, fr[1][0].cam.intrinsics, frame_idx=0),
           Request(1, 100, 0.0, odd, fr[1][0].cam.intrinsics, frame_idx=100)]
    srv = Server(P, budget_bytes=4 << 30, max_batch=8, n_lanes=2, max_w=1280, max_h=720)
    out = srv.run(reqs + bad, realtime=False)
    srv.close()
    assert srv.stats['invalid'] == 3
    for r in bad:
        assert r.refused and r.error and r.planes is None
    assert 'intrinsics' in bad[0].error and 'outside' in bad[1].error
    assert 'changed its frame size' in bad[2].error
    good = [r for r in out if r.error is None]
    assert len(good) == len(reqs) and all(r.planes is not None for r in good)
    ref = alone(fr, good)
    for r in good:
        assert np.array_equal(r.planes.planes, ref[(r.stream, r.k)].planes)
    s = summarize(out, srv.elapsed)
    assert s['invalid'] == 3 and s['frames'] == len(reqs)


def test_admission_is_bounded_by_the_memory_budget():
    fr, host = pool(2, 1)
    reqs = make_reqs(fr, host, [(s, k, 0.0) for k in range(3) for s in range(2)], 1)
    probe = Server(P, budget_bytes=8 << 30, max_batch=4, n_lanes=1)
    one = max(probe.request_bytes(r) for r in reqs)
    static = probe.static_bytes
    probe.close()
    buffers = sum(2 * r.depth.numel() * r.depth.element_size()
                  for r in {r.stream: r for r in reqs}.values())
    srv = Server(P, budget_bytes=static + buffers + one + 1024, max_batch=4, n_lanes=1)
    out = srv.run(reqs, realtime=False)
    srv.close()
    assert all(r.t_done is not None for r in out)
    assert srv.stats['peak_in_use'] <= one + 1024
    assert srv.stats['batches'] == len(reqs)          # one request fits at a time


def test_tuner_keeps_results_bit_identical():
    frames = [synth.frame_c4(7, i) for i in range(4)]
    mw, mh = max(f.w for f in frames), max(f.h for f in frames)
    dev = [torch.from_numpy(f.encoded).cuda() for f in frames]
    batch = [dict(depth=dev[i], K=f.cam.intrinsics, frame_idx=i, iters=f.meta['iters'])
             for i, f in enumerate(frames)]
    with Pipeline(P, mw, mh, len(frames)) as pipe:
        before = pipe.process_batch(batch, use_graph=False)
        res = DiffusionTuner(candidates=[(4, 48, 24), (8, 80, 48), (6, 64, 32)], reps=1).tune(
            pipe, batch)
        assert res['best'] in [(4, 48, 24), (8, 80, 48), (6, 64, 32)]
        after = pipe.process_batch(batch, use_graph=True)
    for a, b in zip(before, after):
        assert np.array_equal(a.planes, b.planes)
