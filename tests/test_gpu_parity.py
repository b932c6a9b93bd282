"""GPU parity: every libpm entry point against the FP64 oracle on the same
seeded inputs, plus form-equivalence (temporal blocking, batch vs single,
graph vs stream launches, host vs device entry).

Tolerances (the targets, written here):
  diffusion            <= 1e-5 m max abs (FP32 and FP16-storage paths alike)
  normals              <= 0.05 deg
  plane normal/offset  <= 0.1 deg / 1 mm
  inlier labels        bit-exact (the inlier decision is FP32 on both sides)
"""
import ctypes
import functools

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2411_01919_b300 import Params, Pipeline, PmError
from e2e_check import chain_job, check_chain, check_end_to_end, oracle_chain

pytestmark = pytest.mark.gpu

DIFF_TOL = 1e-5
NORMAL_TOL_DEG = 0.05
PLANE_DEG, PLANE_OFF = 0.1, 1e-3
DEV = 'cuda:0'


def F32(x):
    """A parameter as the library receives it (the C ABI carries FP32)."""
    return float(np.float32(x))


LAM, KC, SCALE = F32(0.2), F32(0.02), F32(0.001)

CFG = {
    'c1': dict(frame=lambda s: synth.frame_c1(s), iters=10, H=256, max_planes=4),
    'c2': dict(frame=lambda s: synth.frame_c2(s), iters=30, H=1024, max_planes=12),
    'c3': dict(frame=lambda s: synth.frame_c3(s), iters=40, H=2048, max_planes=16),
}


@functools.lru_cache(maxsize=None)
def frame(name, seed=0):
    return CFG[name]['frame'](seed)


def params(name, **kw):
    c = CFG[name]
    p = Params(iters=c['iters'], hypotheses=c['H'], max_planes=c['max_planes'],
               min_inliers=100, seed=11)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def ang_deg(a, b):
    c = np.clip(np.abs(np.sum(a * b, axis=0)), 0.0, 1.0)
    return np.degrees(np.arccos(c))


# ---------------------------------------------------------------------------
# diffusion (Eq. 1, Alg. 1)
# ---------------------------------------------------------------------------

@functools.lru_cache(maxsize=None)
def oracle_diffused(name, mode=0, seed=0):
    fr = frame(name, seed)
    return oracle.diffuse(oracle.decode(fr.encoded, fr.dtype, SCALE), CFG[name]['iters'], LAM, KC,
                          mode)


@pytest.mark.parametrize('name', ['c1', 'c2', 'c3'])
@pytest.mark.parametrize('mode', [0, 1])
def test_diffuse_matches_oracle(name, mode):
    fr = frame(name)
    p = params(name, mode=mode)
    with Pipeline(p, fr.w, fr.h) as pipe:
        z = pipe.diffuse(to_dev(fr.encoded)).cpu().numpy().astype(np.float64)
    ref = oracle_diffused(name, mode)
    err = np.abs(z - ref).max()
    print('%s mode %d: max |gpu - oracle| = %.3e m' % (name, mode, err))
    assert err <= DIFF_TOL
    assert np.array_equal(z == 0, ref == 0)


def _random_depth(h, w, seed, holes=0.05, dtype='f32'):
    rng = np.random.default_rng(seed)
    z = 1.0 + 0.5 * rng.random() + 0.01 * rng.standard_normal((h, w))
    z += 0.1 * (np.arange(w)[None, :] > w // 3)
    z[rng.random((h, w)) < holes] = 0.0
    enc = {'f32': z.astype(np.float32), 'f16': z.astype(np.float16),
           'u16': np.rint(z * 1000).astype(np.uint16)}[dtype]
    return enc


@pytest.mark.parametrize('shape', [(1, 1), (1, 37), (37, 1), (33, 65), (97, 129), (200, 3),
                                   (31, 300)])
@pytest.mark.parametrize('dtype', ['f32', 'u16', 'f16'])
@pytest.mark.parametrize('T', [0, 1, 3])
def test_diffuse_ragged_shapes(shape, dtype, T):
    h, w = shape
    enc = _random_depth(h, w, h * 1000 + w, dtype=dtype)
    p = Params(iters=13, iters_per_launch=T)
    with Pipeline(p, w, h) as pipe:
        z = pipe.diffuse(to_dev(enc)).cpu().numpy().astype(np.float64)
    ref = oracle.diffuse(oracle.decode(enc, dtype, SCALE), 13, LAM, KC, 0)
    assert np.abs(z - ref).max() <= DIFF_TOL


def test_diffuse_all_holes_and_zero_iterations():
    enc = np.zeros((40, 50), dtype=np.float32)
    with Pipeline(Params(iters=5), 50, 40) as pipe:
        assert torch.count_nonzero(pipe.diffuse(to_dev(enc))).item() == 0
    enc = _random_depth(40, 50, 3)
    with Pipeline(Params(iters=0), 50, 40) as pipe:
        z = pipe.diffuse(to_dev(enc)).cpu().numpy()
    assert np.array_equal(z, np.where(enc > 0, enc, 0))


@pytest.mark.parametrize('mode', [0, 1])
def test_temporal_blocking_is_bit_exact(mode):
    fr = frame('c2')
    outs = []
    for T, tw, th in ((1, 0, 0), (2, 0, 0), (3, 0, 0), (5, 0, 0), (8, 0, 0), (8, 80, 48),
                      (8, 48, 24), (7, 17, 9), (4, 64, 1), (8, 1, 48), (6, 33, 40),
                      (4, 122, 32), (8, 128, 48),
                      # (PM4) the register-blocked kernel's (128 - 2T) x (8R - 2T) tiles
                      (8, 112, 48), (8, 112, 32), (8, 112, 16), (6, 116, 36), (4, 120, 56),
                      (3, 122, 26), (1, 126, 62), (2, 124, 44), (5, 118, 22), (7, 114, 50)):
        p = params('c2', mode=mode, iters_per_launch=T, tile_w=tw, tile_h=th)
        with Pipeline(p, fr.w, fr.h) as pipe:
            outs.append(pipe.diffuse(to_dev(fr.encoded)).cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint32), outs[0].view(np.uint32))


@pytest.mark.parametrize('dtype', ['f32', 'u16', 'f16'])
@pytest.mark.parametrize('shape,pad', [((97, 130), 0), ((64, 256), 0), ((64, 256), 3),
                                       ((5, 1029), 1), ((300, 7), 0), ((37, 280), 0),
                                       ((200, 640), 0), ((3, 512), 8)])
@pytest.mark.parametrize('mode', [0, 1])
def test_one_iteration_kernel_is_bit_exact_on_every_encoding(dtype, shape, pad, mode):
    """The streaming kernel against the tiled kernel, bit for bit, on every
    encoding: rows staged in shared memory by asynchronous copies on whole,
    aligned strips (256 x 37 and 512 x 3 of a 280- / 520-wide row: one ring
    strip and a ragged one), vector loads in registers when only the row
    pitch allows, element loads otherwise."""
    h, w = shape
    enc = _random_depth(h, w, 7 * h + w, dtype=dtype)
    wide = np.zeros((h, w + pad), dtype=enc.dtype)
    wide[:, :w] = enc
    d = to_dev(wide)[:, :w]
    outs = []
    for T, tw, th in ((1, 0, 0), (0, 0, 0), (5, 0, 0), (5, 48, 24), (5, 118, 38), (4, 120, 24)):
        with Pipeline(Params(iters=11, mode=mode, iters_per_launch=T, tile_w=tw, tile_h=th),
                      w, h) as pipe:
            outs.append(pipe.diffuse(d).cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint32), outs[0].view(np.uint32))
    ref = oracle.diffuse(oracle.decode(enc, dtype, SCALE), 11, LAM, KC, mode)
    assert np.abs(outs[0].astype(np.float64) - ref).max() <= DIFF_TOL


def test_fp16_storage_path_within_bar():
    fr = frame('c3')
    with Pipeline(params('c3'), fr.w, fr.h) as pipe:
        z = pipe.diffuse(to_dev(fr.encoded)).cpu().numpy().astype(np.float64)
    err = np.abs(z - oracle_diffused('c3')).max()
    assert err <= 5e-4 and err <= DIFF_TOL


# ---------------------------------------------------------------------------
# normals (Eq. 2 reading, Alg. 1 second loop)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize('name', ['c1', 'c2', 'c3'])
@pytest.mark.parametrize('stencil', [0, 1])
def test_normals_match_oracle(name, stencil):
    fr = frame(name)
    z32 = oracle_diffused(name).astype(np.float32)
    with Pipeline(params(name, stencil=stencil), fr.w, fr.h) as pipe:
        P, N, V = pipe.normals(to_dev(z32), fr.cam.intrinsics)
        P, N, V = P.cpu().numpy(), N.cpu().numpy(), V.cpu().numpy()
    Po, No, Vo = oracle.normals(z32.astype(np.float64), fr.cam.intrinsics, stencil)
    assert np.array_equal(V, Vo)
    ok = (V & 2) > 0
    err = ang_deg(N[:, ok].astype(np.float64), No[:, ok]).max()
    print('%s stencil %d: normals max angle %.2e deg over %d px' % (name, stencil, err, ok.sum()))
    assert err <= NORMAL_TOL_DEG
    assert np.abs(P.astype(np.float64) - Po).max() <= 1e-5


@pytest.mark.parametrize('stencil', [0, 1])
@pytest.mark.parametrize('shape', [(480, 640), (37, 61), (5, 130), (64, 4)])
def test_normals_vector_and_element_paths_are_bit_identical(shape, stencil):
    """The normals kernel reads and writes 4 pixels with 16-byte accesses when
    the width is a multiple of 4 and the arrays are aligned, with element
    accesses otherwise: a depth image one float off 16-byte alignment takes
    the element path, and both give the same bits; ragged widths (element
    path) against the oracle."""
    h, w = shape
    rng = np.random.default_rng(h * 7 + w)
    z = (1.0 + 0.3 * rng.random((h, w)) + 0.002 * np.arange(w)[None, :]).astype(np.float32)
    z[rng.random((h, w)) < 0.03] = 0.0
    K = (0.9 * w, 0.9 * w, w / 2.0, h / 2.0)
    with Pipeline(params('c1', stencil=stencil), w, h) as pipe:
        a = [t.cpu().numpy() for t in pipe.normals(to_dev(z), K)]
        buf = torch.zeros(h * w + 1, dtype=torch.float32, device=DEV)
        buf[1:] = to_dev(z).reshape(-1)
        b = [t.cpu().numpy() for t in pipe.normals(buf[1:].view(h, w), K)]
    for x, y in zip(a, b):
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8))
    Po, No, Vo = oracle.normals(z.astype(np.float64), K, stencil)
    assert np.array_equal(a[2], Vo)
    ok = (a[2] & 2) > 0
    if ok.any():
        assert ang_deg(a[1][:, ok].astype(np.float64), No[:, ok]).max() <= NORMAL_TOL_DEG


@functools.lru_cache(maxsize=None)
def high_noise(mode):
    """Three times the noise of the 640x480 workload (sigma = 0.006 z^2)."""
    fr = synth.frame_straight(5, 640, 480, 0.006)
    ref = oracle.diffuse(oracle.decode(fr.encoded, fr.dtype, SCALE), 40, LAM, KC, mode)
    return fr, ref


@pytest.mark.parametrize('mode', [0, 1])
@pytest.mark.parametrize('stencil', [0, 1])
def test_high_noise_forty_iterations(mode, stencil):
    """Sec. IV-B: more than 20 diffusion iterations for noisier depth.  Both
    diffusion forms, both normal stencils, 40 iterations at three times the
    workload's noise, against the oracle."""
    fr, ref = high_noise(mode)
    p = Params(iters=40, mode=mode, stencil=stencil)
    with Pipeline(p, fr.w, fr.h) as pipe:
        z = pipe.diffuse(to_dev(fr.encoded)).cpu().numpy().astype(np.float64)
        z32 = ref.astype(np.float32)
        P, N, V = pipe.normals(to_dev(z32), fr.cam.intrinsics)
        N, V = N.cpu().numpy(), V.cpu().numpy()
    err = np.abs(z - ref).max()
    print('high noise mode %d: max |gpu - oracle| = %.3e m' % (mode, err))
    assert err <= DIFF_TOL
    assert np.array_equal(z == 0, ref == 0)
    Po, No, Vo = oracle.normals(z32.astype(np.float64), fr.cam.intrinsics, stencil)
    assert np.array_equal(V, Vo)
    ok = (V & 2) > 0
    assert ang_deg(N[:, ok].astype(np.float64), No[:, ok]).max() <= NORMAL_TOL_DEG


# ---------------------------------------------------------------------------
# RANSAC (Eq. 3, Alg. 2), same FP32 points on both sides
# ---------------------------------------------------------------------------

@functools.lru_cache(maxsize=None)
def ransac_inputs(name):
    fr = frame(name)
    P, N, V = oracle.normals(oracle_diffused(name), fr.cam.intrinsics, 0)
    return P.astype(np.float32), N.astype(np.float32), V


@functools.lru_cache(maxsize=None)
def oracle_ransac(name, frame_idx=0):
    P, N, V = ransac_inputs(name)
    p = params(name)
    return oracle.ransac(P, N, V, p.hypotheses, p.thr, p.max_planes, p.min_inliers, p.seed,
                         p.gate_deg, frame_idx)


def compare_planes(gpu, orc, exact_labels=True):
    assert len(gpu.planes) == len(orc.planes)
    assert np.array_equal(gpu.hyp_index, orc.hyp_index)
    assert np.array_equal(gpu.n_inliers, orc.n_inliers)
    for k in range(len(orc.planes)):
        a, b = gpu.planes[k], orc.planes[k]
        assert ang_deg(a[:3, None], b[:3, None])[0] <= PLANE_DEG
        assert abs(a[3] - b[3]) <= PLANE_OFF
        assert a[3] > 0
    # the refit gate is the same FP32 decision on both sides
    assert np.array_equal(gpu.n_refit, orc.n_refit)


@pytest.mark.parametrize('name', ['c1', 'c2', 'c3'])
def test_ransac_stage_bit_exact_labels(name):
    fr = frame(name)
    P, N, V = ransac_inputs(name)
    orc = oracle_ransac(name)
    with Pipeline(params(name), fr.w, fr.h) as pipe:
        g = pipe.ransac_planes(to_dev(P), to_dev(N), to_dev(V), frame_idx=0)
        lab = g.labels.cpu().numpy()
    print('%s: %d planes, near-threshold band counts %s' % (name, len(orc.planes), orc.band))
    compare_planes(g, orc)
    assert np.array_equal(lab, orc.labels)


def test_ransac_to_the_plane_limit():
    """64 sequential rounds (the plane limit) on a uniform random cloud, where
    every round finds a plane through a few dozen points: labels, winners
    and counts equal the oracle's in every round."""
    rng = np.random.default_rng(7)
    h, w = 40, 50
    P = rng.uniform(-0.5, 0.5, (3, h, w)).astype(np.float32)
    P[2] += 2.0
    V = np.ones((h, w), dtype=np.uint8)
    p = Params(iters=0, hypotheses=64, max_planes=64, min_inliers=3, seed=5)
    orc = oracle.ransac(P, None, V, p.hypotheses, p.thr, p.max_planes, p.min_inliers, p.seed,
                        p.gate_deg, 3)
    assert len(orc.planes) == 64
    with Pipeline(p, w, h) as pipe:
        pipe.set_timing(2)
        g = pipe.ransac_planes(to_dev(P), None, to_dev(V), frame_idx=3)
        lab = g.labels.cpu().numpy()
        st = pipe.kernel_stats()
    assert np.array_equal(g.hyp_index, orc.hyp_index)
    assert np.array_equal(g.n_inliers, orc.n_inliers)
    assert np.array_equal(lab, orc.labels)
    assert st['score_launches'] == 64 and st['score_pairs'] > 0


def test_ransac_single_hypothesis_per_round():
    fr = frame('c1')
    P, N, V = ransac_inputs('c1')
    p = Params(iters=0, hypotheses=1, max_planes=8, min_inliers=3, seed=5)
    orc = oracle.ransac(P, N, V, p.hypotheses, p.thr, p.max_planes, p.min_inliers, p.seed,
                        p.gate_deg, 3)
    with Pipeline(p, fr.w, fr.h) as pipe:
        g = pipe.ransac_planes(to_dev(P), to_dev(N), to_dev(V), frame_idx=3)
        lab = g.labels.cpu().numpy()
    compare_planes(g, orc)
    assert np.array_equal(lab, orc.labels)


def test_ransac_frame_index_changes_hypotheses():
    fr = frame('c1')
    P, N, V = ransac_inputs('c1')
    orc = oracle_ransac('c1', 5)
    with Pipeline(params('c1'), fr.w, fr.h) as pipe:
        g = pipe.ransac_planes(to_dev(P), to_dev(N), to_dev(V), frame_idx=5)
        assert np.array_equal(g.labels.cpu().numpy(), orc.labels)
    compare_planes(g, orc)


def test_ransac_without_normals_uses_all_inliers():
    fr = frame('c1')
    P, _, V = ransac_inputs('c1')
    p = params('c1')
    orc = oracle.ransac(P, None, V, p.hypotheses, p.thr, p.max_planes, p.min_inliers, p.seed,
                        p.gate_deg, 0)
    with Pipeline(p, fr.w, fr.h) as pipe:
        g = pipe.ransac_planes(to_dev(P), None, to_dev(V), frame_idx=0)
        assert np.array_equal(g.labels.cpu().numpy(), orc.labels)
    compare_planes(g, orc)
    assert np.array_equal(g.n_refit, orc.n_refit)


def threshold_slab_scene(z0, half_w, thr, h=64, w=128):
    """Points on the plane z = z0 (rows 0-39) and pairs of rows offset along
    z by thr (1 -/+ 2^-22), above or below, just inside or just outside the
    threshold: each two-row strip of the candidate order is eight whole
    32-point segments (16 x 2 pixels) whose boxes lie at the threshold
    distance from planes near z = z0."""
    xs = np.linspace(-half_w, half_w, w, dtype=np.float64)
    ys = np.linspace(-0.6 * half_w, 0.6 * half_w, h, dtype=np.float64)
    X, Y = np.meshgrid(xs, ys)
    Z = np.full((h, w), z0, dtype=np.float64)
    t32 = float(np.float32(thr))
    for v in range(40, h):
        k = (v - 40) // 2                          # the strip
        sign = 1.0 if k % 2 == 0 else -1.0          # above / below the plane
        rel = (1.0 - 2.0 ** -22) if (k // 2) % 2 == 0 else (1.0 + 2.0 ** -22)
        Z[v, :] = z0 + sign * t32 * rel
    P = np.stack([X, Y, Z]).astype(np.float32)
    V = np.ones((h, w), dtype=np.uint8)
    return P, V


@pytest.mark.parametrize('z0,half_w', [(1.5, 0.5), (9.5, 6.0)])
def test_box_culling_keeps_threshold_inliers(z0, half_w):
    """The scoring kernel skips pairs by a box test; segments that sit at the
    threshold distance from the winning plane must be decided exactly as
    the oracle (which evaluates every pair) decides them."""
    thr = 0.01
    P, V = threshold_slab_scene(z0, half_w, thr)
    h, w = V.shape
    # seed: one whose winning hypotheses have points at the threshold in both scenes
    p = Params(iters=0, hypotheses=512, thr=thr, max_planes=2, min_inliers=50, seed=50)
    orc = oracle.ransac(P, None, V, p.hypotheses, p.thr, p.max_planes, p.min_inliers, p.seed,
                        p.gate_deg, 0)
    with Pipeline(p, w, h) as pipe:
        g = pipe.ransac_planes(to_dev(P), None, to_dev(V), frame_idx=0)
        lab = g.labels.cpu().numpy()
    assert np.array_equal(g.hyp_index, orc.hyp_index)
    assert np.array_equal(g.n_inliers, orc.n_inliers)
    assert np.array_equal(lab, orc.labels)
    # the scene does put points of the winning plane within 1e-6 m of the
    # threshold, where a box test without a sound margin would drop inliers
    assert orc.band[0] > 0


@pytest.mark.parametrize('z0,w,h', [(1.25, 61, 37), (7.0, 100, 41)])
def test_box_inclusion_counts_whole_segments(z0, w, h):
    """Every point on the plane z = z0, a candidate count that is not a
    multiple of the 32-point segment: every hypothesis through three
    non-collinear points is the plane itself, its slab holds every segment's
    box, and the scoring kernel adds whole (and the ragged last) segments
    without evaluating a pair.  Counts, winner and labels equal the oracle's."""
    xs = np.linspace(-0.4, 0.4, w)
    ys = np.linspace(-0.3, 0.3, h)
    X, Y = np.meshgrid(xs, ys)
    P = np.stack([X, Y, np.full((h, w), z0)]).astype(np.float32)
    V = np.ones((h, w), dtype=np.uint8)
    p = Params(iters=0, hypotheses=256, thr=0.01, max_planes=2, min_inliers=50, seed=9)
    orc = oracle.ransac(P, None, V, p.hypotheses, p.thr, p.max_planes, p.min_inliers, p.seed,
                        p.gate_deg, 0)
    with Pipeline(p, w, h) as pipe:
        pipe.set_timing(2)
        g = pipe.ransac_planes(to_dev(P), None, to_dev(V), frame_idx=0)
        lab = g.labels.cpu().numpy()
        st = pipe.kernel_stats()
    assert (w * h) % 32 != 0
    assert np.array_equal(g.hyp_index, orc.hyp_index)
    assert np.array_equal(g.n_inliers, orc.n_inliers) and g.n_inliers[0] == w * h
    assert np.array_equal(lab, orc.labels)
    assert st['score_pairs'] >= p.hypotheses * w * h
    assert st['evaluated_pairs'] == 0


# ---------------------------------------------------------------------------
# the whole path
# ---------------------------------------------------------------------------

@pytest.mark.parametrize('name', ['c1', 'c2', 'c3'])
def test_process_frame_matches_oracle(name):
    """The whole path on one frame, stage by stage with teacher forcing (each
    oracle stage on the GPU's output of the stage before: e2e_check), plus the
    structural comparison with the oracle's own chain."""
    fr = frame(name)
    p = params(name)
    out = torch.empty((fr.h, fr.w), dtype=torch.float32, device=DEV)
    lab = torch.empty((fr.h, fr.w), dtype=torch.int16, device=DEV)
    with Pipeline(p, fr.w, fr.h) as pipe:
        g = pipe.process_batch([dict(depth=to_dev(fr.encoded), K=fr.cam.intrinsics, frame_idx=0,
                                     labels=lab, depth_out=out)], use_graph=False)[0]
        P, N, V = (t.cpu().numpy() for t in pipe.frame_geometry(0, fr.w, fr.h))
        single = pipe.process_frame(to_dev(fr.encoded), fr.cam.intrinsics, frame_idx=0)
    job = chain_job(fr, p, p.iters, 0, out.cpu().numpy(), P, N, V)
    r = oracle_chain(job)
    n = check_chain(r, g, lab.cpu().numpy(), DIFF_TOL, name)
    print('%s: %d planes equal to the oracle stage by stage; diffusion %.2e m, normals %.2e deg'
          % (name, n, r['diff_err'], r['normal_err']))
    if name != 'c3':
        res = oracle.process_frame(fr.encoded, fr.dtype, fr.cam.intrinsics, p.iters, LAM, KC,
                                   hypotheses=p.hypotheses, max_planes=p.max_planes,
                                   min_inliers=p.min_inliers, seed=p.seed, frame_idx=0,
                                   depth_scale=SCALE)
        agree = check_end_to_end(fr, g, lab.cpu().numpy(), res.ransac,
                                 min_big=300 if name == 'c1' else 2000)
        print('%s: own-chain oracle %d planes, surface agreement %.5f'
              % (name, len(res.ransac.planes), agree))
    assert np.array_equal(single.planes, g.planes)
    assert np.array_equal(single.labels.cpu().numpy(), lab.cpu().numpy())


# ---------------------------------------------------------------------------
# forms: batch vs single, graph vs stream launches, host vs device
# ---------------------------------------------------------------------------

def test_batch_and_graph_equal_single_frames():
    frames = [synth.frame_c4(3, i) for i in range(5)] + [frame('c1'), frame('c2')]
    p = Params(iters=25, hypotheses=512, max_planes=6, min_inliers=100, seed=3)
    mw = max(f.w for f in frames)
    mh = max(f.h for f in frames)
    dev = [to_dev(f.encoded) for f in frames]
    iters = [f.meta.get('iters', 25) for f in frames]
    with Pipeline(p, mw, mh, len(frames)) as pipe:
        singles = []
        for i, f in enumerate(frames):
            pipe1 = Pipeline(Params(**{**p.__dict__, 'iters': iters[i]}), mw, mh, 1)
            singles.append(pipe1.process_frame(dev[i], f.cam.intrinsics, frame_idx=100 + i))
            pipe1.close()
        for use_graph in (False, True, True):
            labs = [torch.empty((f.h, f.w), dtype=torch.int16, device=DEV) for f in frames]
            res = pipe.process_batch([dict(depth=dev[i], K=f.cam.intrinsics, frame_idx=100 + i,
                                           iters=iters[i], labels=labs[i])
                                      for i, f in enumerate(frames)], use_graph=use_graph)
            for i in range(len(frames)):
                assert np.array_equal(res[i].planes, singles[i].planes)
                assert np.array_equal(res[i].n_inliers, singles[i].n_inliers)
                assert torch.equal(labs[i], singles[i].labels)


def test_odd_sized_batch_stage_by_stage_and_alone():
    """Frames of odd width and height in one batch: the candidate order's last
    strip is a single row and every frame ends in a ragged chunk.  Each frame
    is checked stage by stage against the oracle (teacher forcing: every plane
    round's winner, counts and labels exactly) and equals the frame alone."""
    sizes = [(641, 479), (333, 211), (197, 123)]
    frames = [synth.frame_straight(40 + i, w, h) for i, (w, h) in enumerate(sizes)]
    p = Params(iters=20, hypotheses=512, max_planes=8, min_inliers=100, seed=5)
    mw, mh = max(w for w, _ in sizes), max(h for _, h in sizes)
    dev = [to_dev(f.encoded) for f in frames]
    with Pipeline(p, mw, mh, len(frames)) as pipe:
        labs = [torch.empty((f.h, f.w), dtype=torch.int16, device=DEV) for f in frames]
        outs = [torch.empty((f.h, f.w), dtype=torch.float32, device=DEV) for f in frames]
        res = pipe.process_batch([dict(depth=dev[i], K=f.cam.intrinsics, frame_idx=7 + i,
                                       labels=labs[i], depth_out=outs[i])
                                  for i, f in enumerate(frames)], use_graph=True)
        geo = [[t.cpu().numpy() for t in pipe.frame_geometry(i, f.w, f.h)]
               for i, f in enumerate(frames)]
        singles = [pipe.process_frame(dev[i], f.cam.intrinsics, frame_idx=7 + i)
                   for i, f in enumerate(frames)]
    for i, f in enumerate(frames):
        assert np.array_equal(res[i].planes, singles[i].planes)
        assert torch.equal(labs[i], singles[i].labels)
        job = chain_job(f, p, p.iters, 7 + i, outs[i].cpu().numpy(), *geo[i])
        n = check_chain(oracle_chain(job), res[i], labs[i].cpu().numpy(), DIFF_TOL,
                        '%dx%d' % (f.w, f.h))
        assert n >= 2


def test_resume_in_a_fresh_context_is_bit_identical():
    """The only state of a stream is (seed, frame index): a frame processed
    again in a new context, after other frames went through the old one,
    gives bit-identical planes and labels."""
    fr = frame('c2')
    p = params('c2')
    d = to_dev(fr.encoded)
    with Pipeline(p, fr.w, fr.h) as pipe:
        a = pipe.process_frame(d, fr.cam.intrinsics, frame_idx=41)
        la = a.labels.cpu().numpy()
        for i in range(3):
            pipe.process_frame(to_dev(frame('c2', i + 1).encoded), fr.cam.intrinsics, frame_idx=i)
    with Pipeline(p, fr.w, fr.h) as pipe:
        b = pipe.process_frame(d, fr.cam.intrinsics, frame_idx=41)
        lb = b.labels.cpu().numpy()
    assert np.array_equal(a.planes.view(np.uint64), b.planes.view(np.uint64))
    assert np.array_equal(a.hyp_index, b.hyp_index) and np.array_equal(la, lb)


def test_hypotheses_drawn_in_compaction_equal_separate_launch():
    """A context whose frames may exceed 4096 chunks draws each round's
    hypotheses in a launch of their own from the compacted list; a smaller
    one draws them inside the compaction from the list being compacted.
    Both give the same hypotheses, so planes, winners and labels agree bit
    for bit (single frame and a batch)."""
    frames = [frame('c2'), synth.frame_c4(7, 0), synth.frame_c4(7, 1)]
    p = Params(iters=20, hypotheses=700, max_planes=8, min_inliers=100, seed=11)
    mw = max(f.w for f in frames)
    mh = max(f.h for f in frames)
    dev = [to_dev(f.encoded) for f in frames]
    assert mw * mh <= 4096 * 1024 < 2048 * 2049
    out = []
    for w, h in ((mw, mh), (2048, 2049)):
        with Pipeline(p, w, h, len(frames)) as pipe:
            one = pipe.process_frame(dev[0], frames[0].cam.intrinsics, frame_idx=5)
            labs = [torch.empty((f.h, f.w), dtype=torch.int16, device=DEV) for f in frames]
            res = pipe.process_batch([dict(depth=dev[i], K=f.cam.intrinsics, frame_idx=5 + i,
                                           labels=labs[i]) for i, f in enumerate(frames)])
            out.append((one.planes.copy(), one.hyp_index.copy(), one.labels.cpu().numpy(),
                        [(r.planes.copy(), r.hyp_index.copy()) for r in res],
                        [l.cpu().numpy() for l in labs]))
    a, b = out
    assert len(a[0]) >= 3
    assert np.array_equal(a[0].view(np.uint64), b[0].view(np.uint64))
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    for (pa, ha), (pb, hb) in zip(a[3], b[3]):
        assert np.array_equal(pa.view(np.uint64), pb.view(np.uint64)) and np.array_equal(ha, hb)
    for la, lb in zip(a[4], b[4]):
        assert np.array_equal(la, lb)


def test_host_entry_equals_device_entry():
    fr = frame('c2')
    p = params('c2')
    with Pipeline(p, fr.w, fr.h) as pipe:
        d = pipe.process_frame(to_dev(fr.encoded), fr.cam.intrinsics, frame_idx=9)
        lab = np.empty((fr.h, fr.w), dtype=np.int16)
        h = pipe.process_frame_host(fr.encoded, fr.cam.intrinsics, frame_idx=9, labels=lab)
    assert np.array_equal(d.planes, h.planes)
    assert np.array_equal(d.labels.cpu().numpy(), lab)


def test_host_batch_entry_equals_device_batch():
    """pm_process_batch_host_async (depth in pinned or pageable host memory,
    copied by the call) gives the device batch's results bit for bit, with
    and without graph replay."""
    frames = [synth.frame_c4(5, i) for i in range(6)]
    p = Params(iters=20, hypotheses=512, max_planes=6, min_inliers=100, seed=4)
    mw, mh = max(f.w for f in frames), max(f.h for f in frames)

    def desc(depths):
        return [dict(depth=depths[i], K=f.cam.intrinsics, frame_idx=50 + i, iters=f.meta['iters'])
                for i, f in enumerate(frames)]

    with Pipeline(p, mw, mh, len(frames)) as pipe:
        ref = pipe.process_batch(desc([to_dev(f.encoded) for f in frames]), use_graph=False)
        pinned = [torch.from_numpy(f.encoded).pin_memory() for f in frames]
        for depths, use_graph in ((pinned, False), (pinned, True), (pinned, True),
                                  ([f.encoded for f in frames], True)):
            pipe.submit_batch_host(desc(depths), use_graph=use_graph)
            torch.cuda.synchronize()
            got = pipe.collect_batch()
            for a, b in zip(got, ref):
                assert np.array_equal(a.planes.view(np.uint64), b.planes.view(np.uint64))
                assert np.array_equal(a.hyp_index, b.hyp_index)
                assert np.array_equal(a.n_inliers, b.n_inliers)


# ---------------------------------------------------------------------------
# degenerate inputs and argument errors
# ---------------------------------------------------------------------------

def test_degenerate_frames():
    p = Params(iters=3, hypotheses=64, max_planes=3, min_inliers=10)
    K = (50.0, 50.0, 10.0, 10.0)
    with Pipeline(p, 64, 64) as pipe:
        z = torch.zeros((20, 20), dtype=torch.float32, device=DEV)
        r = pipe.process_frame(z, K)
        assert len(r.planes) == 0 and bool((r.labels == -1).all())
        z = torch.zeros((20, 20), dtype=torch.float32, device=DEV)
        z[5, 5] = 1.0
        z[6, 6] = 1.1
        r = pipe.process_frame(z, K)
        assert len(r.planes) == 0
        z = torch.full((1, 64), 1.5, dtype=torch.float32, device=DEV)
        r = pipe.process_frame(z, K)
        assert len(r.planes) == 0
        f = synth.plane_frame(64, 64, 50.0, 50.0, 31.5, 31.5, [0.2, -0.5, -1.0], 1.2)
        r = pipe.process_frame(to_dev(f.encoded), f.cam.intrinsics)
        assert len(r.planes) == 1
        assert ang_deg(r.planes[0, :3, None], f.planes[0, :3, None])[0] < 0.01
        assert abs(r.planes[0, 3] - f.planes[0, 3]) < 1e-4


def test_argument_errors_raise():
    with Pipeline(Params(iters=2), 32, 32) as pipe:
        with pytest.raises(PmError):
            pipe.diffuse(torch.zeros((40, 40), dtype=torch.float32, device=DEV))
        with pytest.raises(ValueError):
            pipe.diffuse(torch.zeros((4, 4), dtype=torch.float64, device=DEV))
        with pytest.raises(PmError):
            pipe.process_batch([dict(depth=torch.zeros((4, 4), device=DEV), K=(0, 1, 0, 0))])


@pytest.mark.parametrize('ipl', [0, 1])
def test_calls_on_the_scratch_refuse_while_a_batch_is_pending(ipl):
    """While a batch from the asynchronous entry point may still be running,
    every call that would write the context's scratch returns PM_ERR_STATE
    (the one-iteration diffusion path included) and launches nothing."""
    from paper_2411_01919_b300 import _ffi
    fr = frame('c1')
    p = params('c1', iters_per_launch=ipl)
    with Pipeline(p, fr.w, fr.h) as pipe:
        d = to_dev(fr.encoded)
        z0 = pipe.diffuse(d).clone()
        pipe.submit_batch([dict(depth=d, K=fr.cam.intrinsics, frame_idx=3)])
        calls = [lambda: pipe.diffuse(d),
                 lambda: pipe.process_frame_host(fr.encoded, fr.cam.intrinsics),
                 lambda: pipe.process_frame(d, fr.cam.intrinsics),
                 lambda: pipe.frame_geometry(0, fr.w, fr.h)]
        for call in calls:
            with pytest.raises(PmError) as e:
                call()
            assert e.value.status == _ffi.PM_ERR_STATE
        torch.cuda.synchronize()
        got = pipe.collect_batch()[0]
        ref = pipe.process_frame(d, fr.cam.intrinsics, frame_idx=3)
        assert np.array_equal(got.planes, ref.planes)
        assert torch.equal(pipe.diffuse(d), z0)


def test_scratch_allocation_failure_is_reported_and_recoverable():
    """A context whose scratch cannot be allocated (about 22 TB) returns
    PM_ERR_OOM -- an ordinary allocation failure, nothing launched -- and the
    device stays usable for the next context."""
    from paper_2411_01919_b300 import _ffi
    with pytest.raises(PmError) as ei:
        Pipeline(Params(iters=2), 16000, 16000, 1024)
    assert ei.value.status == _ffi.PM_ERR_OOM
    fr = frame('c1')
    with Pipeline(params('c1'), fr.w, fr.h) as pipe:
        r = pipe.process_frame(to_dev(fr.encoded), fr.cam.intrinsics)
    assert len(r.planes) >= 1


def test_misaligned_device_pointers_are_rejected_before_launch():
    """A device buffer not aligned to its element size is refused on the host
    (PM_ERR_ARG) before any kernel could touch it."""
    from paper_2411_01919_b300 import _ffi
    buf = torch.zeros(32 * 32 + 4, dtype=torch.float32, device=DEV)
    out = torch.zeros(32 * 32 + 4, dtype=torch.float32, device=DEV)
    base, obase = buf.data_ptr(), out.data_ptr()
    with Pipeline(Params(iters=2), 32, 32) as pipe:
        lib, h = pipe.lib, pipe._h
        assert lib.pm_diffuse(h, base + 2, _ffi.PM_F32_M, 32, 32, 128, obase, None) == _ffi.PM_ERR_ARG
        assert lib.pm_diffuse(h, base + 1, _ffi.PM_U16_MM, 32, 32, 64, obase, None) == _ffi.PM_ERR_ARG
        assert lib.pm_diffuse(h, base, _ffi.PM_F32_M, 32, 32, 128, obase + 2, None) == _ffi.PM_ERR_ARG
        assert b'align' in lib.pm_last_error()
        K = _ffi.Intrinsics(30.0, 30.0, 16.0, 16.0)
        planes = (_ffi.Plane * 4)()
        n = ctypes.c_int(0)
        st = lib.pm_process_frame(h, base, _ffi.PM_F32_M, 32, 32, 128, ctypes.byref(K), 0, planes,
                                  4, ctypes.byref(n), obase + 1, None)
        assert st == _ffi.PM_ERR_ARG
        # the aligned call goes through
        assert lib.pm_diffuse(h, base, _ffi.PM_F32_M, 32, 32, 128, obase, None) == _ffi.PM_OK
        torch.cuda.synchronize()


def test_graph_replay_records_kernel_timing_events():
    fr = frame('c1')
    p = params('c1')
    d = to_dev(fr.encoded)
    with Pipeline(p, fr.w, fr.h, 2) as pipe:
        pipe.set_timing(2)
        batch = [dict(depth=d, K=fr.cam.intrinsics, frame_idx=i) for i in range(2)]
        for s in (None, torch.cuda.Stream()):
            with torch.cuda.stream(s or torch.cuda.current_stream()):
                pipe.process_batch(batch, use_graph=True)       # capture
                pipe.process_batch(batch, use_graph=True)       # replay
            st = pipe.kernel_stats()
            assert st['score_ms'] > 0 and st['score_pairs'] > 0
            assert 0 < st['evaluated_pairs'] <= st['score_pairs']
            assert st['launches'] >= 3 + 3 * p.max_planes
