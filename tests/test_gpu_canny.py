"""GPU parity of the Canny edges of the normal image and of the regions they
bound, against the oracle.  Every decision is integer (8-bit codes from one
FP32 FMA on both sides, integer Sobel, exact sector test, union-find
components), so edges and region labels are compared bit-exactly."""
import ctypes
import functools

import numpy as np
import pytest
import torch
from scipy import ndimage

import oracle
import synth
from paper_2411_01919_b300 import Params, Pipeline, PmError

pytestmark = pytest.mark.gpu

DEV = 'cuda:0'


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@functools.lru_cache(maxsize=None)
def staircase_normals(name):
    fr = {'c1': synth.frame_c1, 'c2': synth.frame_c2, 'c3': synth.frame_c3}[name](0)
    iters = {'c1': 10, 'c2': 30, 'c3': 40}[name]
    z = oracle.decode(fr.encoded, fr.dtype)
    zs = oracle.diffuse(z, iters, 0.2, 0.02, 0)
    P, N, V = oracle.normals(zs, fr.cam.intrinsics, 0)
    return N.astype(np.float32), V, fr


def gpu_edges(N, V, low, high):
    _, h, w = N.shape
    with Pipeline(Params(iters=0), w, h, 1) as pipe:
        return pipe.canny(to_dev(N), to_dev(V), low, high).cpu().numpy()


def gpu_segment(E, V, min_pixels, gap):
    h, w = E.shape
    with Pipeline(Params(iters=0), w, h, 1) as pipe:
        lab, R = pipe.segment(to_dev(E), to_dev(V), min_pixels, gap)
        return lab.cpu().numpy(), R


@pytest.mark.parametrize('name', ['c1', 'c2', 'c3'])
@pytest.mark.parametrize('low,high', [(60, 150), (20, 40), (150, 400)])
def test_canny_bit_exact_on_staircases(name, low, high):
    N, V, _ = staircase_normals(name)
    want = oracle.canny(N, V, low, high)
    got = gpu_edges(N, V, low, high)
    assert np.array_equal(got, want)
    assert want.sum() > 0


def smooth_normals(h, w, seed, holes=0.03):
    rng = np.random.default_rng(seed)
    N = rng.normal(0, 1, (3, h, w))
    N = ndimage.gaussian_filter(N, (0, 2.0, 2.0))
    N /= np.linalg.norm(N, axis=0, keepdims=True)
    V = (rng.random((h, w)) > holes).astype(np.uint8)
    return N.astype(np.float32), V


@pytest.mark.parametrize('shape', [(1, 1), (1, 37), (37, 1), (2, 2), (33, 65), (97, 129),
                                   (8, 32), (9, 33), (200, 3)])
def test_canny_ragged_shapes(shape):
    h, w = shape
    N, V = smooth_normals(h, w, h * 1000 + w)
    for low, high in ((0, 0), (40, 120), (100, 300)):
        assert np.array_equal(gpu_edges(N, V, low, high), oracle.canny(N, V, low, high))


def test_canny_all_invalid_and_constant():
    N = np.zeros((3, 20, 30), np.float32)
    N[2] = -1
    V = np.zeros((20, 30), np.uint8)
    assert gpu_edges(N, V, 0, 0).sum() == 0
    V[:] = 1
    assert gpu_edges(N, V, 0, 0).sum() == 0


@pytest.mark.parametrize('name', ['c1', 'c2', 'c3'])
@pytest.mark.parametrize('gap,min_pixels', [(1, 200), (0, 1), (1, 1), (0, 50)])
def test_segment_bit_exact_on_staircase_edges(name, gap, min_pixels):
    N, V, _ = staircase_normals(name)
    E = oracle.canny(N, V)
    want, R = oracle.segment(E, V, min_pixels, gap)
    got, Rg = gpu_segment(E, V, min_pixels, gap)
    assert Rg == R
    assert np.array_equal(got, want)


@pytest.mark.parametrize('seed,shape,density', [(0, (1, 1), 0.0), (1, (1, 50), 0.2),
                                                (2, (50, 1), 0.2), (3, (61, 97), 0.05),
                                                (4, (61, 97), 0.3), (5, (300, 257), 0.1)])
def test_segment_random_edge_masks(seed, shape, density):
    rng = np.random.default_rng(seed)
    E = (rng.random(shape) < density).astype(np.uint8)
    V = (rng.random(shape) > 0.05).astype(np.uint8)
    for gap in (0, 1):
        for mp in (1, 7):
            want, R = oracle.segment(E, V, mp, gap)
            got, Rg = gpu_segment(E, V, mp, gap)
            assert Rg == R and np.array_equal(got, want)


def test_segment_one_region_spanning_the_image():
    """A spiral-free serpentine: one 4-connected region that winds through the
    whole image (long union-find chains)."""
    h, w = 128, 256
    E = np.zeros((h, w), np.uint8)
    for r in range(2, h - 2, 4):
        E[r, (0 if (r // 4) % 2 else 2):(w - 2 if (r // 4) % 2 else w)] = 1
    V = np.ones((h, w), np.uint8)
    want, R = oracle.segment(E, V, 1, 0)
    got, Rg = gpu_segment(E, V, 1, 0)
    assert R == Rg == 1 and np.array_equal(got, want)


def test_edges_regions_planes_chain_on_the_gpu():
    """Normals, edges, regions and per-region RANSAC all on the GPU: the
    regions lie on single ground-truth planes and the large ones are
    accepted with the right normal."""
    fr = synth.frame_c1(0)
    p = Params(iters=10, hypotheses=256, thr=0.01, max_planes=4, seed=3)
    with Pipeline(p, fr.w, fr.h, 1) as pipe:
        z = pipe.diffuse(to_dev(fr.encoded))
        P, N, V = pipe.normals(z, fr.cam.intrinsics)
        E = pipe.canny(N, V)
        lab, R = pipe.segment(E, V, 100)
        out = pipe.ransac_regions(P, V, lab, R, 256)
        labn = lab.cpu().numpy()
    assert R >= 4
    for r in range(R):
        ids, cnt = np.unique(fr.plane_id[labn == r], return_counts=True)
        assert cnt.max() >= 0.95 * cnt.sum()
        k = ids[np.argmax(cnt)]
        if out.total[r] >= 1000 and k >= 0:
            assert out.accepted[r]
            n = out.planes[r, :3] / np.linalg.norm(out.planes[r, :3])
            assert np.degrees(np.arccos(min(1.0, abs(float(n @ fr.planes[k, :3]))))) < 5.0


def test_argument_errors_raise():
    N = np.zeros((3, 8, 8), np.float32)
    V = np.ones((8, 8), np.uint8)
    with Pipeline(Params(iters=0), 8, 8, 1) as pipe:
        with pytest.raises(PmError):
            pipe.canny(to_dev(N), to_dev(V), 10, 5)
        with pytest.raises(PmError):
            pipe.segment(to_dev(V), to_dev(V), 0, 1)
        with pytest.raises(PmError):
            pipe.segment(to_dev(V), to_dev(V), 1, 2)
        big = np.zeros((3, 9, 9), np.float32)
        with pytest.raises(PmError):
            pipe.canny(to_dev(big), to_dev(np.ones((9, 9), np.uint8)), 1, 2)


def test_canny_allocates_nothing_and_captures_into_a_graph():
    """The context allocates the edge scratch when it is created, so pm_canny
    can be captured into a CUDA graph on its first call; the replay gives the
    same edges as a direct call."""
    N, V, _ = staircase_normals('c2')
    _, h, w = N.shape
    dN, dV = to_dev(N), to_dev(V)
    with Pipeline(Params(iters=0), w, h, 1) as pipe:
        E = torch.empty((h, w), dtype=torch.uint8, device=DEV)
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                st = pipe.lib.pm_canny(pipe._h, ctypes.c_void_p(dN.data_ptr()),
                                       ctypes.c_void_p(dV.data_ptr()), w, h, 60, 150,
                                       ctypes.c_void_p(E.data_ptr()),
                                       ctypes.c_void_p(s.cuda_stream))
        assert st == 0, pipe.lib.pm_last_error()
        g.replay()
        torch.cuda.synchronize()
        direct = pipe.canny(dN, dV, 60, 150)
        assert torch.equal(E, direct)
    assert np.array_equal(E.cpu().numpy(), oracle.canny(N, V, 60, 150))
