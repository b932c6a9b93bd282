"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every check is a closed form, an
invariant, a special case that reduces to a library routine (numpy's Philox,
numpy.linalg.eigh, numpy's float16 decode), exact geometry of analytic scenes,
or brute force on tiny inputs.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth

LAM, KC = 0.2, 0.02


# ---------------------------------------------------------------------------
# decode
# ---------------------------------------------------------------------------

def test_decode_f16_all_bit_patterns():
    bits = np.arange(65536, dtype=np.uint16).reshape(256, 256)
    got = oracle.decode(bits.view(np.float16), 'f16')
    ref = bits.view(np.float16).astype(np.float64)
    ref = np.where(np.isfinite(ref) & (ref > 0), ref, 0.0)
    assert np.array_equal(got, ref)


def test_decode_u16_scale_and_holes():
    e = np.array([[0, 1, 1000, 65535]], dtype=np.uint16)
    got = oracle.decode(e, 'u16', 0.001)
    assert np.array_equal(got, np.array([[0.0, 0.001, 1.0, 65.535]]))


def test_decode_f32_nonfinite_negative_are_holes():
    e = np.array([[np.nan, -1.0, np.inf, 0.0, 1.5]], dtype=np.float32)
    assert np.array_equal(oracle.decode(e, 'f32'), np.array([[0, 0, 0, 0, 1.5]]))


# ---------------------------------------------------------------------------
# diffusion (Eq. 1, Alg. 1)
# ---------------------------------------------------------------------------

def g(x):
    return math.exp(-(x / KC) ** 2)


@pytest.mark.parametrize('h', [0.003, 0.02, 0.05, -0.01])
def test_pm4_spike_closed_form(h):
    I = np.ones((3, 3))
    I[1, 1] += h
    out = oracle.diffuse(I, 1, LAM, KC, 0)
    assert out[1, 1] == pytest.approx(1 + h - 4 * LAM * g(h) * h, abs=1e-15)
    for (v, u) in [(0, 1), (1, 0), (1, 2), (2, 1)]:
        assert out[v, u] == pytest.approx(1 + LAM * g(h) * h, abs=1e-15)
    for (v, u) in [(0, 0), (0, 2), (2, 0), (2, 2)]:
        assert out[v, u] == 1.0


@pytest.mark.parametrize('h', [0.003, 0.02, -0.04])
def test_alg1_spike_closed_form(h):
    I = np.ones((3, 3))
    I[1, 1] += h
    out = oracle.diffuse(I, 1, LAM, KC, 1)
    # centre: all neighbours equal -> zero gradient, c = 1, Laplacian = -4h
    assert out[1, 1] == pytest.approx(1 + h - 4 * LAM * h, abs=1e-15)
    # edge-centre: one neighbour is the spike; the gradient along that axis is h/2
    c = math.exp(-((abs(h) / 2) / KC) ** 2)
    for (v, u) in [(0, 1), (1, 0), (1, 2), (2, 1)]:
        assert out[v, u] == pytest.approx(1 + LAM * c * h, abs=1e-15)
    for (v, u) in [(0, 0), (0, 2), (2, 0), (2, 2)]:
        assert out[v, u] == 1.0


def _noisy(seed, h=24, w=31, holes=0.1):
    rng = np.random.default_rng(seed)
    I = 1.0 + 0.03 * rng.standard_normal((h, w)) + 0.2 * (np.arange(w) > w // 2)
    I[rng.random((h, w)) < holes] = 0.0
    return I


def test_pm4_conserves_sum_over_valid_pixels():
    I = _noisy(1)
    V = I > 0
    for it in (1, 5, 30):
        out = oracle.diffuse(I, it, LAM, KC, 0)
        assert out[V].sum() == pytest.approx(I[V].sum(), rel=1e-14)


@pytest.mark.parametrize('mode', [0, 1])
def test_maximum_principle(mode):
    I = _noisy(2)
    V = I > 0
    out = oracle.diffuse(I, 25, LAM, KC, mode)
    assert out[V].min() >= I[V].min() - 1e-15
    assert out[V].max() <= I[V].max() + 1e-15
    assert np.all(out[~V] == 0.0)


@pytest.mark.parametrize('mode', [0, 1])
def test_offset_invariance(mode):
    I = _noisy(3)
    V = I > 0
    J = np.where(V, I + 0.75, 0.0)
    a = oracle.diffuse(I, 10, LAM, KC, mode)
    b = oracle.diffuse(J, 10, LAM, KC, mode)
    assert np.max(np.abs(b[V] - 0.75 - a[V])) < 1e-13


@pytest.mark.parametrize('mode', [0, 1])
def test_constant_is_fixed_point(mode):
    I = np.full((9, 13), 1.234)
    assert np.array_equal(oracle.diffuse(I, 7, LAM, KC, mode), I)


def test_pm4_linear_ramp_interior_fixed():
    u = np.arange(20, dtype=np.float64)
    I = np.tile(1.0 + 0.004 * u, (7, 1))
    out = oracle.diffuse(I, 1, LAM, KC, 0)
    # interior columns: the E and W fluxes cancel exactly; the border columns see one flux
    assert np.max(np.abs(out[:, 1:-1] - I[:, 1:-1])) < 1e-15
    assert out[0, 0] > I[0, 0] and out[0, -1] < I[0, -1]


@pytest.mark.parametrize('mode', [0, 1])
def test_flip_and_transpose_symmetry(mode):
    I = _noisy(4)
    a = oracle.diffuse(I, 6, LAM, KC, mode)
    assert np.max(np.abs(oracle.diffuse(I[:, ::-1], 6, LAM, KC, mode) - a[:, ::-1])) < 1e-14
    assert np.max(np.abs(oracle.diffuse(I[::-1, :], 6, LAM, KC, mode) - a[::-1, :])) < 1e-14
    assert np.max(np.abs(oracle.diffuse(I.T, 6, LAM, KC, mode) - a.T)) < 1e-14


@pytest.mark.parametrize('mode', [0, 1])
def test_holes_block_flux(mode):
    # [a, hole, b]: every neighbour of a and b is outside or a hole -> nothing changes
    I = np.array([[1.0, 0.0, 2.0]])
    assert np.array_equal(oracle.diffuse(I, 5, LAM, KC, mode), I)
    # a pixel next to a hole evolves as if the hole carried its own value
    rng = np.random.default_rng(5)
    J = 1 + 0.01 * rng.standard_normal((5, 5))
    J[2, 2] = 0.0
    out = oracle.diffuse(J, 1, LAM, KC, mode)
    assert out[2, 2] == 0.0


def test_diffusion_rejects_unstable_lambda():
    with pytest.raises(ValueError):
        oracle.diffuse(np.ones((4, 4)), 1, 0.3, KC, 0)


# ---------------------------------------------------------------------------
# normals (Eq. 2 reading, Alg. 1 second loop)
# ---------------------------------------------------------------------------

PLANES = [([0.0, 0.0, -1.0], 2.0), ([0.3, -0.8, -0.5], 1.3), ([-0.6, 0.2, -0.7], 0.9),
          ([0.0, -1.0, -0.2], 1.0)]


@pytest.mark.parametrize('stencil', [0, 1])
@pytest.mark.parametrize('n,d', PLANES)
def test_normals_exact_on_analytic_planes(n, d, stencil):
    f = synth.plane_frame(64, 48, 60.0, 62.0, 31.5, 23.0, n, d)
    P, N, V = oracle.normals(f.depth, f.cam.intrinsics, stencil)
    nn = f.planes[0, :3]
    ok = (V & 2) > 0
    assert ok.sum() > 100
    err = np.abs(N[:, ok] - nn[:, None]).max()
    assert err < 1e-12
    # back-projected points lie on the plane
    res = np.einsum('k,kij->ij', nn, P) + f.planes[0, 3]
    assert np.abs(res[(V & 1) > 0]).max() < 1e-12


def test_normals_match_sphere_geometry():
    # camera-frame sphere of radius R centred at C; exact outward normals (P - C)/R
    w, h, fx, fy, cx, cy = 120, 100, 500.0, 500.0, 59.5, 49.5
    C, R = np.array([0.05, -0.03, 3.0]), 1.0
    u, v = np.meshgrid(np.arange(w), np.arange(h))
    dvec = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u, dtype=float)], -1)
    a = (dvec ** 2).sum(-1)
    b = -2 * dvec @ C
    c = C @ C - R * R
    disc = b * b - 4 * a * c
    z = np.where(disc > 0, (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a), 0.0)
    P, N, V = oracle.normals(z, (fx, fy, cx, cy), 0)
    ok = (V & 2) > 0
    exact = (P - C[:, None, None]) / R
    cosang = np.clip((N * exact).sum(0)[ok], -1, 1)
    # central differences are second-order: pixel pitch ~ 4 mm on a 1 m sphere
    assert np.degrees(np.arccos(cosang)).max() < 0.05
    assert ok.sum() > 3000


def test_normals_validity_border_and_holes():
    f = synth.plane_frame(20, 16, 20.0, 20.0, 9.5, 7.5, [0, 0, -1], 1.0)
    z = f.depth.copy()
    z[8, 10] = 0.0
    P, N, V = oracle.normals(z, f.cam.intrinsics, 0)
    assert not (V[0, :] & 2).any() and not (V[-1, :] & 2).any()
    assert not (V[:, 0] & 2).any() and not (V[:, -1] & 2).any()
    assert V[8, 10] == 0 and np.all(P[:, 8, 10] == 0)
    for (vv, uu) in [(7, 10), (9, 10), (8, 9), (8, 11)]:
        assert V[vv, uu] == 1                      # depth valid, normal invalid
    assert V[8, 12] == 3
    P1, N1, V1 = oracle.normals(z, f.cam.intrinsics, 1)
    assert V1[7, 9] == 1 and V1[7, 12] == 3        # Sobel needs all 8 neighbours


# ---------------------------------------------------------------------------
# Philox4x64-10 and the eigen-solver
# ---------------------------------------------------------------------------

def _numpy_philox_block(ctr, key):
    """philox(ctr) via numpy, which outputs philox(counter + 1) first."""
    c = [int(x) for x in ctr]
    val = sum(c[i] << (64 * i) for i in range(4)) - 1
    val %= 1 << 256
    cm1 = np.array([(val >> (64 * i)) & ((1 << 64) - 1) for i in range(4)], dtype=np.uint64)
    b = np.random.Philox(counter=cm1, key=np.array(key, dtype=np.uint64))
    return b.random_raw(4)


@pytest.mark.parametrize('ctr,key', [
    ([0, 0, 0, 0], [0, 0]),
    ([5, 7, 11, 13], [0x0123456789abcdef, 0xfedcba9876543210]),
    ([2**64 - 1, 3, 2**63, 1], [2**64 - 1, 2**64 - 1]),
    ([123, 4, 99, 0], [42, 0]),
])
def test_philox_matches_numpy(ctr, key):
    ctr = np.array(ctr, dtype=np.uint64)
    got = oracle.philox4x64_10(ctr, key)
    assert np.array_equal(got, _numpy_philox_block(ctr, key))


def test_eig3_matches_numpy_eigh():
    rng = np.random.default_rng(0)
    for _ in range(200):
        A = rng.standard_normal((3, 3))
        A = A @ A.T * rng.uniform(1e-6, 10)
        ev, V = oracle.eig3(A)
        rev, rV = np.linalg.eigh(A)
        assert np.allclose(ev, rev, rtol=1e-12, atol=1e-15 * abs(rev).max())
        for k in range(3):
            assert abs(abs(V[:, k] @ rV[:, k]) - 1) < 1e-9
    ev, V = oracle.eig3(np.diag([3.0, 1.0, 2.0]))
    assert np.array_equal(ev, [1.0, 2.0, 3.0])


# ---------------------------------------------------------------------------
# RANSAC (Eq. 3, Alg. 2)
# ---------------------------------------------------------------------------

def _tiny_scene(seed, w=6, h=5):
    """<= 30 points: two planes with small noise plus far outliers."""
    rng = np.random.default_rng(seed)
    n = w * h
    P = np.zeros((3, n))
    kind = rng.integers(0, 3, n)          # 0 floor, 1 wall, 2 outlier
    x = rng.uniform(-0.5, 0.5, n)
    y = rng.uniform(-0.5, 0.5, n)
    P[:, kind == 0] = np.stack([x, np.full(n, 0.8), 2.0 + y])[:, kind == 0]
    P[:, kind == 1] = np.stack([x, y, np.full(n, 2.5)])[:, kind == 1]
    P[:, kind == 2] = np.stack([x, y, 1.5 + rng.uniform(0, 2, n)])[:, kind == 2]
    P += 1e-4 * rng.standard_normal(P.shape)
    valid = np.ones(n, dtype=np.uint8)
    valid[rng.random(n) < 0.1] = 0
    return P.reshape(3, h, w).astype(np.float32), valid.reshape(h, w)


def _strip_candidates(valid):
    """Flat indices of the valid pixels in the candidate order of the RANSAC
    rounds: two-row strips top to bottom, each strip column by column, the
    upper pixel of a column first (one row in the last strip of an odd height)."""
    h, w = valid.shape
    ys, xs = np.mgrid[0:h, 0:w]
    order = np.lexsort((ys.ravel(), xs.ravel(), ys.ravel() // 2))
    return order[(valid.reshape(-1)[order] & 1) > 0]


def test_strip_candidate_order_small_frame():
    # 3 x 3 frame, all valid: strip 0 = rows 0-1 column by column, strip 1 = row 2
    order = _strip_candidates(np.ones((3, 3), np.uint8))
    assert order.tolist() == [0, 3, 1, 4, 2, 5, 6, 7, 8]


def _indices_numpy(seed, frame_idx, r, hyp, M):
    w = _numpy_philox_block(np.array([hyp, r, frame_idx, 0], dtype=np.uint64), [seed, 0])
    return [(int(x) * M) >> 64 for x in w[:3]]


def _count64(pl, Pc, thr):
    res = pl[:3] @ Pc + pl[3]
    return int((np.abs(res) < thr).sum()), np.abs(np.abs(res) - thr).min()


@pytest.mark.parametrize('seed', range(6))
def test_ransac_brute_force_tiny(seed):
    P, valid = _tiny_scene(seed)
    H, thr, seed_rng, frame = 64, 0.01, 1234 + seed, 7
    r = oracle.ransac(P, None, valid, H, thr, 1, 1, seed_rng, 20.0, frame)
    Pf = P.reshape(3, -1).astype(np.float64)
    cand = _strip_candidates(valid)
    M = len(cand)
    Pc = Pf[:, cand]
    checked = 0
    for h in range(H):
        idx = _indices_numpy(seed_rng, frame, 0, h, M)
        q = Pc[:, idx]
        n = np.cross(q[:, 1] - q[:, 0], q[:, 2] - q[:, 0])
        if np.linalg.norm(n) <= 1e-9:
            assert r.counts[0, h] == -1
            continue
        n /= np.linalg.norm(n)
        pl = np.r_[n, -n @ q[:, 0]]
        cnt, margin = _count64(pl, Pc, thr)
        if margin < 1e-5:          # a point within 10 um of the threshold: FP32 may decide otherwise
            continue
        assert r.counts[0, h] == cnt
        checked += 1
    assert checked >= H // 2
    # the winner is the maximum count, ties to the lowest index
    best = int(np.argmax(r.counts[0]))
    assert r.hyp_index[0] == best
    # no triplet at all scores more than what brute force over every triplet allows
    allbest = 0
    for tri in itertools.combinations(range(M), 3):
        q = Pc[:, tri]
        n = np.cross(q[:, 1] - q[:, 0], q[:, 2] - q[:, 0])
        if np.linalg.norm(n) <= 1e-9:
            continue
        n /= np.linalg.norm(n)
        allbest = max(allbest, _count64(np.r_[n, -n @ q[:, 0]], Pc, thr)[0])
    assert r.n_inliers[0] <= allbest
    assert allbest - r.n_inliers[0] <= 2


def test_ransac_labels_are_inliers_of_winner():
    P, valid = _tiny_scene(11, 12, 10)
    r = oracle.ransac(P, None, valid, 128, 0.01, 3, 3, 5, 20.0, 0)
    Pf = P.reshape(3, -1).astype(np.float64)
    lab = r.labels.reshape(-1)
    assert np.all(lab[(valid.reshape(-1) & 1) == 0] == -1)
    for k in range(len(r.planes)):
        sel = lab == k
        assert sel.sum() == r.n_inliers[k]
        pl = r.planes[k]
        assert np.abs(pl[:3] @ Pf[:, sel] + pl[3]).max() < 0.02


@pytest.mark.parametrize('n,d', PLANES[:3])
def test_ransac_recovers_single_analytic_plane(n, d):
    f = synth.plane_frame(80, 60, 70.0, 70.0, 39.5, 29.5, n, d)
    P, N, V = oracle.normals(f.depth, f.cam.intrinsics, 0)
    r = oracle.ransac(P.astype(np.float32), N.astype(np.float32), V, 64, 0.01, 2, 50, 3)
    assert len(r.planes) == 1
    gt = f.planes[0]
    assert np.degrees(np.arccos(min(1.0, r.planes[0, :3] @ gt[:3]))) < 1e-4
    assert abs(r.planes[0, 3] - gt[3]) < 1e-6
    assert r.n_inliers[0] == int((V & 1).sum())
    assert r.rms[0] < 1e-6


def test_ransac_refit_gate_counts_the_normals_within_the_gate():
    """The refit uses the inliers whose normal is valid and within the gate
    angle of the hypothesis normal, in either orientation; with fewer than
    three such inliers it uses them all.  A fronto-parallel plane (every
    hypothesis normal is exactly (0, 0, +-1)) with per-pixel normals tilted by
    known angles, none near the 20 degree boundary, fixes the count."""
    f = synth.plane_frame(40, 30, 35.0, 35.0, 19.5, 14.5, (0.0, 0.0, 1.0), -2.0)
    P, _, V = oracle.normals(f.depth, f.cam.intrinsics, 0)
    V = V.copy()
    h, w = V.shape
    rng = np.random.default_rng(2)
    angles = rng.choice([0.0, 7.0, 19.9, 19.99, 20.01, 20.2, 35.0, 89.0, 160.5, 175.0, 180.0],
                        size=(h, w))
    N = np.stack([np.zeros((h, w)), np.sin(np.radians(angles)), -np.cos(np.radians(angles))])
    V |= 2
    V[rng.random((h, w)) < 0.1] &= 1          # normal invalid: never gated
    within = (np.minimum(angles, 180.0 - angles) < 20.0) & ((V & 2) > 0)
    r = oracle.ransac(P.astype(np.float32), N.astype(np.float32), V, 16, 0.01, 1, 50, 3)
    assert r.n_inliers[0] == h * w
    assert r.n_refit[0] == int(within.sum())
    assert abs(r.planes[0, 2] + 1.0) < 1e-12 and abs(r.planes[0, 3] - 2.0) < 1e-6
    # fewer than three normals within the gate: the refit takes every inlier
    a2 = np.full((h, w), 45.0)
    a2[3, 5] = a2[7, 9] = 0.0
    N2 = np.stack([np.zeros((h, w)), np.sin(np.radians(a2)), -np.cos(np.radians(a2))])
    r = oracle.ransac(P.astype(np.float32), N2.astype(np.float32), V | 2, 16, 0.01, 1, 50, 3)
    assert r.n_refit[0] == h * w
    a2[11, 13] = 180.0                         # a third one, the other way round
    N2 = np.stack([np.zeros((h, w)), np.sin(np.radians(a2)), -np.cos(np.radians(a2))])
    r = oracle.ransac(P.astype(np.float32), N2.astype(np.float32), V | 2, 16, 0.01, 1, 50, 3)
    assert r.n_refit[0] == 3
    r = oracle.ransac(P.astype(np.float32), N.astype(np.float32), V & 1, 16, 0.01, 1, 50, 3)
    assert r.n_refit[0] == h * w


def test_ransac_recovers_noise_free_staircase():
    rng = np.random.Generator(np.random.PCG64(0))
    cam = synth.make_camera(160, 120, 120.0, 120.0, 80.0, 60.0, [0.0, 0.0, 1.0], 0.0, np.pi / 4)
    sc = synth.straight_staircase(3, 0.15, 0.28, 1.0, first_riser_y=0.6)
    fr = synth.sense(sc, cam, rng, 0.0, 0.0, False, 'f32')
    res = oracle.process_frame(fr.encoded, 'f32', cam.intrinsics, iters=0, hypotheses=256,
                               max_planes=8, min_inliers=100, seed=1)
    rr = res.ransac
    assert len(rr.planes) >= 6
    ids, counts = np.unique(fr.plane_id[fr.plane_id >= 0], return_counts=True)
    for k, pl in enumerate(rr.planes):
        sel = rr.labels == k
        gid = np.bincount(fr.plane_id[sel][fr.plane_id[sel] >= 0]).argmax()
        gt = fr.planes[gid]
        assert np.degrees(np.arccos(min(1.0, pl[:3] @ gt[:3]))) < 0.01
        assert abs(pl[3] - gt[3]) < 1e-4
    # every GT plane with more than 3% of the pixels is found
    found = {np.bincount(fr.plane_id[(rr.labels == k) & (fr.plane_id >= 0)]).argmax()
             for k in range(len(rr.planes))}
    for gid, c in zip(ids, counts):
        if c > 0.03 * fr.w * fr.h:
            assert gid in found


def test_ransac_stops_below_min_inliers_and_on_empty():
    P = np.zeros((3, 4, 4), dtype=np.float32)
    valid = np.zeros((4, 4), dtype=np.uint8)
    r = oracle.ransac(P, None, valid, 16, 0.01, 4, 1, 0)
    assert len(r.planes) == 0 and np.all(r.labels == -1)
    Pn, vn = _tiny_scene(3)
    r = oracle.ransac(Pn, None, vn, 16, 0.01, 4, 1000, 0)
    assert len(r.planes) == 0


def test_ransac_deterministic_and_frame_dependent():
    P, valid = _tiny_scene(9, 12, 10)
    a = oracle.ransac(P, None, valid, 64, 0.01, 2, 3, 5, 20.0, 0)
    b = oracle.ransac(P, None, valid, 64, 0.01, 2, 3, 5, 20.0, 0)
    c = oracle.ransac(P, None, valid, 64, 0.01, 2, 3, 5, 20.0, 1)
    assert np.array_equal(a.counts, b.counts) and np.array_equal(a.labels, b.labels)
    assert not np.array_equal(a.counts, c.counts)
