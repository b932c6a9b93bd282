"""GPU parity of per-region RANSAC (Alg. 2 per polygon) against the oracle.

Everything the method decides here is an integer or comes from exactly
specified FP32 operations (the samples' pixels, the hypothesis plane, the
distance sums in units of 2^-32 m, the inlier counts, the argmin and the 90%
acceptance), so the comparison is bit-exact on every field.
"""
import functools

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2411_01919_b300 import Params, Pipeline, PmError

pytestmark = pytest.mark.gpu

DEV = 'cuda:0'
THR = 0.01


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def pipe_for(w, h, seed):
    return Pipeline(Params(iters=0, hypotheses=256, thr=THR, max_planes=4, seed=seed), w, h, 1)


def run_both(P, V, regions, R, H, seed, frame_idx=0):
    P = np.ascontiguousarray(P, dtype=np.float32)
    _, h, w = P.shape
    orc = oracle.ransac_regions(P, V, regions, R, H, THR, seed, frame_idx)
    with pipe_for(w, h, seed) as pipe:
        gpu = pipe.ransac_regions(to_dev(P), to_dev(V.astype(np.uint8)),
                                  to_dev(regions.astype(np.int32)), R, H, frame_idx)
    return gpu, orc


def assert_same(gpu, orc):
    assert np.array_equal(gpu.total, orc.total)
    assert np.array_equal(gpu.hyp_index, orc.hyp_index)
    assert np.array_equal(gpu.error, orc.error)
    assert np.array_equal(gpu.inliers, orc.inliers)
    assert np.array_equal(gpu.accepted, orc.accepted)
    # the stored plane is the FP32 hypothesis of both sides
    assert np.array_equal(gpu.planes, orc.planes)


@functools.lru_cache(maxsize=None)
def staircase_inputs(name):
    fr = {'c1': synth.frame_c1, 'c2': synth.frame_c2}[name](0)
    z = oracle.decode(fr.encoded, fr.dtype)
    zs = oracle.diffuse(z, 10, 0.2, 0.02, 0)
    P, N, V = oracle.normals(zs, fr.cam.intrinsics, 0)
    return P.astype(np.float32), V, fr.plane_id.astype(np.int32), len(fr.planes)


@pytest.mark.parametrize('name,H', [('c1', 64), ('c1', 37), ('c2', 128)])
def test_staircase_regions_bit_exact(name, H):
    P, V, regions, R = staircase_inputs(name)
    gpu, orc = run_both(P, V, regions, R, H, seed=3)
    assert_same(gpu, orc)
    assert gpu.accepted.sum() >= 3


def test_frame_index_changes_the_samples():
    P, V, regions, R = staircase_inputs('c1')
    a, oa = run_both(P, V, regions, R, 32, seed=5, frame_idx=0)
    b, ob = run_both(P, V, regions, R, 32, seed=5, frame_idx=7)
    assert_same(a, oa)
    assert_same(b, ob)
    assert not np.array_equal(a.error, b.error)


def plane_points(h, w, n, d):
    f = synth.plane_frame(w, h, 60.0, 60.0, (w - 1) / 2, (h - 1) / 2, n, d)
    P, N, V = oracle.normals(f.depth, f.cam.intrinsics, 0)
    return P.astype(np.float32), V


def test_outliers_tiny_empty_and_foreign_labels():
    """A clean region, 5% and 20% outlier regions, a non-convex region, a
    two-point region, an empty region and labels outside [0, R)."""
    rng = np.random.default_rng(2)
    P, V = plane_points(48, 64, [0.1, -0.5, -1.0], 1.5)
    P = P.copy()
    regions = np.full((48, 64), -1, dtype=np.int32)
    regions[:24, :20] = 0
    regions[:24, 20:40] = 1
    regions[24:, :40] = 2
    regions[2:22, 44:50] = 3                  # L-shaped
    regions[16:22, 44:62] = 3
    regions[30, 50:52] = 4                    # two points
    regions[40:, 50:] = 9                     # label >= R: ignored
    regions[26:29, 44:47] = -7                # negative label: ignored
    flat = P.reshape(3, -1)
    for r, frac in ((1, 0.05), (2, 0.20)):
        idx = np.flatnonzero(regions.reshape(-1) == r)
        out = rng.choice(idx, int(round(frac * idx.size)), replace=False)
        flat[2, out] += 0.3
    V = V.copy()
    V[3, 3] = 0                               # an invalid point inside region 0
    gpu, orc = run_both(P, V, regions, 6, 48, seed=8)
    assert_same(gpu, orc)
    assert gpu.accepted[0] and gpu.accepted[1] and gpu.accepted[3]
    assert not gpu.accepted[2]
    assert gpu.hyp_index[4] == -1 and gpu.hyp_index[5] == -1 and gpu.total[5] == 0


def test_many_small_regions_and_a_region_over_many_chunks():
    """128 cells of 12x8 pixels plus one big region (several 256-point chunks,
    ragged tail), H not a multiple of the 32-hypothesis block."""
    rng = np.random.default_rng(9)
    P, V = plane_points(96, 160, [0.3, -0.4, -1.0], 1.2)
    P = P + (rng.normal(0, 0.003, P.shape) * (V > 0)).astype(np.float32)
    regions = np.full((96, 160), -1, dtype=np.int32)
    cells = 0
    for cy in range(8):
        for cx in range(16):
            regions[cy * 12:(cy + 1) * 12, cx * 8:(cx + 1) * 8] = cells
            cells += 1
    regions[:, 128:] = cells                  # 96 x 32 = 3072 points: 12 chunks
    V = V.copy()
    V[95, 159] = 0                            # ragged last chunk
    gpu, orc = run_both(P, V, regions, cells + 1, 45, seed=1)
    assert_same(gpu, orc)
    assert gpu.total[cells] == 3071


def test_hypotheses_at_the_limit():
    P, V = plane_points(40, 56, [0.0, -0.6, -1.0], 1.3)
    regions = np.zeros((40, 56), dtype=np.int32)
    regions[:, 28:] = 1
    gpu, orc = run_both(P, V, regions, 2, 2048, seed=4)
    assert_same(gpu, orc)


def test_all_points_invalid():
    P, V = plane_points(16, 24, [0.0, -0.6, -1.0], 1.3)
    V = np.zeros_like(V)
    regions = np.zeros((16, 24), dtype=np.int32)
    gpu, orc = run_both(P, V, regions, 3, 16, seed=0)
    assert_same(gpu, orc)
    assert (gpu.hyp_index == -1).all() and (gpu.total == 0).all()


def test_argument_errors_raise():
    P, V = plane_points(16, 24, [0.0, -0.6, -1.0], 1.3)
    regions = to_dev(np.zeros((16, 24), dtype=np.int32))
    Pd, Vd = to_dev(P), to_dev(V.astype(np.uint8))
    with pipe_for(24, 16, 0) as pipe:
        for R, H in ((0, 16), (65536, 1), (1, 0), (1, 2049), (4096, 2048)):
            with pytest.raises(PmError):
                pipe.ransac_regions(Pd, Vd, regions, R, H)
        # the context is still usable after refused calls
        out = pipe.ransac_regions(Pd, Vd, regions, 1, 16)
        assert out.total[0] == int((V & 1).sum())
