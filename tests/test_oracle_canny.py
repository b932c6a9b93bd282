"""Pins of the oracle's Canny edges on the normal image and of the regions
they bound (Sec. III-D: edge detection on the normal vector image, then the
planar regions).

Checked against: step edges whose Sobel response and thinned position are
known by hand, the direction sector against atan2, the hysteresis against
scipy.ndimage.label, straight boundaries at many angles (thin, on the line),
and the regions against scipy.ndimage.label with 4-connectivity.
"""
import math

import numpy as np
import pytest
from scipy import ndimage

import oracle
import synth

N1 = np.array([0.0, -0.6, -0.8])
N2 = np.array([0.8, 0.0, -0.6])


def two_plane_normals(h, w, mask):
    """Normal image: N2 where mask, N1 elsewhere (FP32 SoA)."""
    N = np.where(mask[None], N2[:, None, None], N1[:, None, None]).astype(np.float32)
    return N, np.ones((h, w), dtype=np.uint8)


def test_constant_normals_have_no_edges():
    N, V = two_plane_normals(20, 30, np.zeros((20, 30), bool))
    assert oracle.canny(N, V, 0, 0).sum() == 0


@pytest.mark.parametrize('k', [1, 7, 15, 28])
def test_vertical_step_gives_one_pixel_edge_left_of_the_step(k):
    """A step between columns k-1 and k: Sobel |gx| = 4 |dq| on both columns,
    0 elsewhere; non-maximum suppression keeps the left one of the equal pair."""
    h, w = 12, 30
    mask = np.zeros((h, w), bool)
    mask[:, k:] = True
    N, V = two_plane_normals(h, w, mask)
    E = oracle.canny(N, V, 10, 20)
    expect = np.zeros((h, w), np.uint8)
    expect[:, k - 1] = 1
    assert np.array_equal(E, expect)


@pytest.mark.parametrize('k', [1, 9, 18])
def test_horizontal_step_gives_one_pixel_edge_above_the_step(k):
    h, w = 20, 25
    mask = np.zeros((h, w), bool)
    mask[k:, :] = True
    N, V = two_plane_normals(h, w, mask)
    E = oracle.canny(N, V, 10, 20)
    expect = np.zeros((h, w), np.uint8)
    expect[k - 1, :] = 1
    assert np.array_equal(E, expect)


def test_thresholds_are_strict_on_the_sobel_magnitude():
    """Step of code difference dq in one channel: m = 4 dq at the step."""
    h, w = 8, 16
    N = np.zeros((3, h, w), np.float32)
    N[2] = -1.0
    # channel 0: codes 128 and 128 + 10 (n = 10 / 127.5 exactly representable enough)
    N[0, :, 8:] = np.float32(10.25 / 127.5)
    V = np.ones((h, w), np.uint8)
    q = np.floor(np.float32(N[0, 0, 9]) * np.float32(127.5) + np.float32(128))
    m = 4 * int(q - 128)
    assert oracle.canny(N, V, m - 1, m - 1).sum() == h
    assert oracle.canny(N, V, m, m).sum() == 0            # m > high is strict
    assert oracle.canny(N, V, m - 1, m).sum() == 0        # weak only: no strong seed


def test_sector_matches_atan2():
    rng = np.random.default_rng(0)
    g = rng.integers(-1020, 1021, size=(20000, 2))
    g = np.concatenate([g, [[5, 0], [0, 5], [-5, 0], [0, -7], [3, 3], [3, -3], [0, 0]]])
    for gx, gy in g:
        s = oracle.canny_sector(gx, gy)
        if gx == 0 and gy == 0:
            assert s == 3
            continue
        a = math.degrees(math.atan2(abs(gy), abs(gx)))       # in [0, 90]
        if a < 22.5:
            want = 0
        elif a > 67.5:
            want = 2
        else:
            want = 1 if gx * gy > 0 else 3
        assert s == want, (gx, gy, a)


def noisy_normals(h, w, seed):
    rng = np.random.default_rng(seed)
    N = rng.normal(0, 1, (3, h, w))
    N = ndimage.gaussian_filter(N, (0, 3.0, 3.0))
    N /= np.linalg.norm(N, axis=0, keepdims=True)
    V = np.ones((h, w), dtype=np.uint8)
    return N.astype(np.float32), V


@pytest.mark.parametrize('seed', [0, 1, 2])
def test_hysteresis_equals_component_labelling(seed):
    N, V = noisy_normals(60, 80, seed)
    E, st = oracle.canny(N, V, 120, 300, states=True)
    lab, n = ndimage.label(st >= 1, structure=np.ones((3, 3)))
    seeds = np.unique(lab[st == 2])
    want = np.isin(lab, seeds[seeds > 0])
    assert np.array_equal(E.astype(bool), want)
    assert 0 < E.sum() < (st >= 1).sum()              # some weak pixels are dropped


@pytest.mark.parametrize('deg', [3, 17, 30, 44, 46, 61, 80, 97, 120, 135, 160, 178])
def test_straight_boundaries_are_thin_and_on_the_line(deg):
    h, w = 64, 64
    th = math.radians(deg)
    dirv = np.array([math.cos(th), math.sin(th)])
    nrm = np.array([-dirv[1], dirv[0]])
    vv, uu = np.mgrid[0:h, 0:w]
    c = np.array([31.3, 32.6])
    dist = (uu - c[0]) * nrm[0] + (vv - c[1]) * nrm[1]
    N, V = two_plane_normals(h, w, dist > 0)
    E = oracle.canny(N, V, 60, 150)
    ys, xs = np.nonzero(E[2:-2, 2:-2])
    d = np.abs((xs + 2 - c[0]) * nrm[0] + (ys + 2 - c[1]) * nrm[1])
    assert len(d) > 40
    assert d.max() <= 1.5
    # thin: across the line, at most two edge pixels per row (steep lines) or column
    steep = abs(dirv[1]) >= abs(dirv[0])
    per = np.bincount(ys if steep else xs)
    assert per.max() <= 2
    # and it is a boundary: the two sides stay apart in the regions
    lab, R = oracle.segment(E, V, 20)
    side = dist > 0
    for r in range(R):
        m = lab == r
        assert side[m].all() or (~side[m]).all()


def test_holes_are_ringed_by_edges():
    h, w = 30, 30
    N, V = two_plane_normals(h, w, np.zeros((h, w), bool))
    V[14:16, 10:12] = 0
    E = oracle.canny(N, V, 60, 150)
    ys, xs = np.nonzero(E)
    assert len(ys) > 0
    assert (np.abs(ys - 14.5) <= 3).all() and (np.abs(xs - 10.5) <= 3).all()


def canonical_scipy(eligible, min_pixels):
    lab, n = ndimage.label(eligible)          # default structure: 4-connectivity
    out = np.full(eligible.shape, -1, np.int32)
    flat = lab.reshape(-1)
    firsts = {}
    for p in np.flatnonzero(flat):
        firsts.setdefault(flat[p], p)
    sizes = np.bincount(flat)
    R = 0
    for comp in sorted(firsts, key=lambda c: firsts[c]):
        if sizes[comp] >= min_pixels:
            out.reshape(-1)[flat == comp] = R
            R += 1
    return out, R


@pytest.mark.parametrize('seed,gap,min_pixels', [(0, 0, 1), (1, 0, 5), (2, 1, 1), (3, 1, 12)])
def test_segment_equals_scipy_labelling(seed, gap, min_pixels):
    rng = np.random.default_rng(seed)
    h, w = 50, 70
    E = (rng.random((h, w)) < 0.12).astype(np.uint8)
    V = (rng.random((h, w)) > 0.05).astype(np.uint8)
    lab, R = oracle.segment(E, V, min_pixels, gap)
    blocked = ndimage.binary_dilation(E > 0, np.ones((3, 3))) if gap else E > 0
    want, Rw = canonical_scipy((V > 0) & ~blocked, min_pixels)
    assert R == Rw
    assert np.array_equal(lab, want)


def test_staircase_regions_are_pure():
    """On the small staircase the regions left by the edges each lie on one
    ground-truth plane."""
    fr = synth.frame_c1(0)
    z = oracle.decode(fr.encoded, fr.dtype)
    zs = oracle.diffuse(z, 10, 0.2, 0.02, 0)
    P, N, V = oracle.normals(zs, fr.cam.intrinsics, 0)
    E = oracle.canny(N.astype(np.float32), V)
    lab, R = oracle.segment(E, V, 100)
    assert R >= 4
    for r in range(R):
        ids, cnt = np.unique(fr.plane_id[lab == r], return_counts=True)
        assert cnt.max() >= 0.97 * cnt.sum()
