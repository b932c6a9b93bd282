"""Parity at the benchmark's full sizes and launch configuration.

The batched forms run as the benchmark runs them (64 frames per batch,
graph-captured, tuned tiling for the 640x480 step); sampled frames of each
batch are checked against the FP64 oracle one by one: diffused depth within
1e-5 m everywhere, and the planes end to end as e2e_check describes.
"""
import functools

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2411_01919_b300 import Params, Pipeline
from e2e_check import check_end_to_end

pytestmark = pytest.mark.gpu

F32 = lambda x: float(np.float32(x))
DIFF_TOL = 1e-5


def check_frame(fr, iters, p, depth_gpu, planes_gpu, labels_gpu, frame_idx):
    res = oracle.process_frame(fr.encoded, fr.dtype, fr.cam.intrinsics, iters, F32(p.lam),
                               F32(p.K), hypotheses=p.hypotheses, thr=p.thr,
                               max_planes=p.max_planes, min_inliers=p.min_inliers, seed=p.seed,
                               gate_deg=p.gate_deg, frame_idx=frame_idx,
                               depth_scale=F32(p.depth_scale))
    err = np.abs(depth_gpu.astype(np.float64) - res.depth).max()
    assert err <= DIFF_TOL, err
    check_end_to_end(fr, planes_gpu, labels_gpu, res.ransac)
    return err


def run_batch(frames, p, iters, use_graph=True, tune=False):
    dev = [torch.from_numpy(f.encoded).cuda() for f in frames]
    outs = [torch.empty((f.h, f.w), dtype=torch.float32, device='cuda') for f in frames]
    labs = [torch.empty((f.h, f.w), dtype=torch.int16, device='cuda') for f in frames]
    mw, mh = max(f.w for f in frames), max(f.h for f in frames)
    batch = [dict(depth=dev[i], K=f.cam.intrinsics, frame_idx=1000 + i, iters=iters[i],
                  depth_out=outs[i], labels=labs[i]) for i, f in enumerate(frames)]
    with Pipeline(p, mw, mh, len(frames)) as pipe:
        if tune:
            from paper_2411_01919_b300.tune import DiffusionTuner
            DiffusionTuner(reps=1).tune(pipe, batch)
        pipe.process_batch(batch, use_graph=use_graph)          # capture
        res = pipe.process_batch(batch, use_graph=use_graph)    # replay
    return res, [o.cpu().numpy() for o in outs], [l.cpu().numpy() for l in labs]


def test_batched_640x480_step_as_benchmarked():
    frames = [synth.frame_c2(s) for s in range(64)]
    p = Params(iters=30, hypotheses=1024, max_planes=12, min_inliers=100, seed=0)
    res, depth, labs = run_batch(frames, p, [30] * 64, tune=True)
    for i in (0, 37, 63):
        check_frame(frames[i], 30, p, depth[i], res[i], labs[i], 1000 + i)


def test_batched_mixed_resolution_64_frames():
    frames = [synth.frame_c4(11, i) for i in range(64)]
    iters = [f.meta['iters'] for f in frames]
    p = Params(iters=30, hypotheses=1024, max_planes=12, min_inliers=100, seed=2)
    res, depth, labs = run_batch(frames, p, iters)
    sizes = {}
    for i, f in enumerate(frames):
        sizes.setdefault((f.w, f.h), i)
    for (w, h), i in sorted(sizes.items())[:3]:
        check_frame(frames[i], iters[i], p, depth[i], res[i], labs[i], 1000 + i)


def test_precision_form_848x480_fp16():
    frames = [synth.frame_c3(s) for s in range(4)]
    p = Params(iters=40, hypotheses=2048, max_planes=16, min_inliers=100, seed=5)
    res, depth, labs = run_batch(frames, p, [40] * 4)
    err = check_frame(frames[1], 40, p, depth[1], res[1], labs[1], 1001)
    assert err <= 5e-4
