"""The bounds-checking build (libpm_bounds.so, PM_DEBUG_BOUNDS), the stand-in
for a memory sanitizer: the whole path on ragged shapes, every diffusion
kernel, odd pitches and a mixed batch gives exactly the release library's
results, and no instrumented access fell outside its buffer."""
import ctypes
import os

import numpy as np
import pytest
import torch

import synth
from paper_2411_01919_b300 import Params, Pipeline, _ffi
from paper_2411_01919_b300.build import LIB_BOUNDS

pytestmark = pytest.mark.gpu


def status(lib):
    v = ctypes.c_ulonglong(0)
    st = lib.pm_debug_bounds(ctypes.byref(v))
    return st, v.value


def ragged(h, w, seed, dtype):
    rng = np.random.default_rng(seed)
    z = 1.2 + 0.3 * rng.random() + 0.01 * rng.standard_normal((h, w))
    z[rng.random((h, w)) < 0.05] = 0.0
    return {'f32': z.astype(np.float32), 'f16': z.astype(np.float16),
            'u16': np.rint(z * 1000).astype(np.uint16)}[dtype]


def test_release_build_reports_it_has_no_checks():
    st, v = status(_ffi.load())
    assert st == _ffi.PM_ERR_STATE and v == 0


def test_bounds_build_matches_release_with_no_violation():
    assert os.path.exists(LIB_BOUNDS), 'build libpm_bounds.so (build(bounds=True))'
    lib = _ffi.load(LIB_BOUNDS)
    assert status(lib) == (_ffi.PM_OK, 0)
    K = (60.0, 60.0, 30.0, 20.0)
    cases = [((1, 1), 'f32', 0), ((37, 1), 'u16', 0), ((33, 65), 'f16', 3), ((97, 129), 'u16', 1),
             ((200, 3), 'f32', 2), ((61, 300), 'u16', 0)]
    for (h, w), dtype, pad in cases:
        enc = ragged(h, w, h * 7 + w, dtype)
        wide = np.zeros((h, w + pad), dtype=enc.dtype)
        wide[:, :w] = enc
        d = torch.from_numpy(wide).cuda()[:, :w]
        for T, tw, th in ((1, 0, 0), (0, 0, 0), (3, 17, 9), (5, 118, 22), (8, 112, 48)):
            p = Params(iters=9, iters_per_launch=T, tile_w=tw, tile_h=th, hypotheses=64,
                       max_planes=3, min_inliers=10)
            outs = []
            for path in (None, LIB_BOUNDS):
                with Pipeline(p, w, h, lib_path=path) as pipe:
                    z = pipe.diffuse(d)
                    P, N, V = pipe.normals(z, K)
                    pl = pipe.process_frame(d, K, frame_idx=3)
                    outs.append((z.cpu().numpy(), N.cpu().numpy(), pl.planes, pl.labels.cpu().numpy()))
            for a, b in zip(*outs):
                assert np.array_equal(a, b)
            assert status(lib) == (_ffi.PM_OK, 0), ((h, w), dtype, (T, tw, th))
    # a mixed-resolution batch through both scoring forms
    frames = [synth.frame_c4(9, i) for i in range(5)]
    mw, mh = max(f.w for f in frames), max(f.h for f in frames)
    p = Params(iters=20, hypotheses=256, max_planes=4, min_inliers=100, seed=1)
    res = []
    for path in (None, LIB_BOUNDS):
        with Pipeline(p, mw, mh, len(frames), lib_path=path) as pipe:
            r = pipe.process_batch([dict(depth=torch.from_numpy(f.encoded).cuda(), K=f.cam.intrinsics,
                                         frame_idx=i, iters=f.meta['iters'])
                                    for i, f in enumerate(frames)], use_graph=True)
            res.append([x.planes for x in r])
    for a, b in zip(*res):
        assert np.array_equal(a, b)
    assert status(lib) == (_ffi.PM_OK, 0)
