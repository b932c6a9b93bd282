"""Host logic of the request loop (no GPU): the admission-time validation that
refuses a request the lanes cannot serve, and the latency summary."""
import math

import torch

from paper_2411_01919_b300.serve import Request, Server, summarize

K = (385.0, 385.0, 320.0, 240.0)


def bare_server(max_w=640, max_h=480):
    """A Server with no lanes: only the host-side state validation reads."""
    s = Server.__new__(Server)
    s.max_w, s.max_h = max_w, max_h
    s.dev = {}
    return s


def req(depth, K=K, stream=0, iters=-1):
    return Request(stream, 0, 0.0, depth, K, frame_idx=0, iters=iters)


def test_valid_requests_pass():
    s = bare_server()
    for dt in (torch.uint16, torch.float16, torch.float32):
        assert s.invalid(req(torch.zeros((480, 640), dtype=dt))) is None
    assert s.invalid(req(torch.zeros((1, 1)))) is None


def test_each_rule_refuses_with_its_reason():
    s = bare_server()
    cases = [
        (req(torch.zeros((480, 641))), 'outside'),
        (req(torch.zeros((481, 640))), 'outside'),
        (req(torch.zeros((0, 640))), 'outside'),
        (req(torch.zeros((4, 4, 3))), '2-D'),
        (req(torch.zeros((4, 4), dtype=torch.float64)), '2-D'),
        (req(torch.zeros((8, 8))[:, ::2]), 'contiguous'),
        (req(torch.zeros((4, 4)), K=(0.0, 385.0, 1.0, 1.0)), 'intrinsics'),
        (req(torch.zeros((4, 4)), K=(385.0, -1.0, 1.0, 1.0)), 'intrinsics'),
        (req(torch.zeros((4, 4)), K=(385.0, 385.0, math.nan, 1.0)), 'intrinsics'),
        (req(torch.zeros((4, 4)), K=(385.0, 385.0, 1.0)), 'four numbers'),
        (req(torch.zeros((4, 4)), iters=100001), 'iters'),
    ]
    for r, why in cases:
        msg = s.invalid(r)
        assert msg is not None and why in msg, (why, msg)


def test_a_stream_keeps_its_frame_size_and_type():
    s = bare_server()
    s.dev[3] = [torch.zeros((240, 424), dtype=torch.uint16)]
    assert s.invalid(req(torch.zeros((240, 424), dtype=torch.uint16), stream=3)) is None
    assert 'changed' in s.invalid(req(torch.zeros((240, 420), dtype=torch.uint16), stream=3))
    assert 'changed' in s.invalid(req(torch.zeros((240, 424), dtype=torch.float16), stream=3))
    assert s.invalid(req(torch.zeros((480, 640)), stream=4)) is None     # another stream


def test_summary_counts_and_percentiles():
    rs = []
    for i in range(101):
        r = req(torch.zeros((2, 2)))
        r.t_arrival, r.t_done = 0.0, i * 1e-3           # latencies 0 .. 100 ms
        rs.append(r)
    bad = req(torch.zeros((2, 2)))
    bad.refused, bad.error = True, 'intrinsics must be finite with fx, fy > 0'
    late = req(torch.zeros((2, 2)))
    late.refused = True
    lost = req(torch.zeros((2, 2)))
    lost.refused, lost.failed, lost.error = True, True, 'batch failed: PM_ERR_CUDA'
    s = summarize(rs + [bad, late, lost], elapsed=2.0)
    assert s['frames'] == 101 and s['refused'] == 3 and s['invalid'] == 1 and s['failed'] == 1
    assert s['p50_ms'] == 50.0 and s['p99_ms'] == 99.0 and s['max_ms'] == 100.0
    assert s['frames_per_s'] == 50.5
