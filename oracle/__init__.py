"""FP64 CPU oracle for the depth -> diffusion -> normals -> planes hot path.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product path (the CUDA library and
its Python binding) never imports this package.

The arithmetic lives in oracle.c (plain C, FP64, inlier decisions in FP32);
this module marshals numpy arrays through ctypes and chains the stages.

Parity status per function (what pins it is listed in the test suite):
  decode          pinned (numpy float16 decode, u16 scale)
  diffuse         pinned (closed-form 3x3 stencils, conservation, maximum
                  principle, offset invariance, fixed points, symmetry, holes)
  normals         pinned (analytic planes to 1e-12, closed-form derivative normal)
  philox4x64_10   pinned (numpy.random.Philox raw output)
  eig3            pinned (numpy.linalg.eigh)
  ransac          pinned (brute force over all triplets on <= 30 points,
                  exact counts of given hypotheses, noise-free staircase planes)
  ransac_regions  pinned (sample uniformity and region membership, FP64 brute-force
                  distance sums per hypothesis, argmin rule, acceptance on single-
                  and two-plane regions, ground-truth planes of a staircase)
  canny           pinned (step edges of known position and width, sector test
                  against atan2, hysteresis against scipy.ndimage.label, edges of
                  straight lines at many angles are thin and on the line)
  segment         pinned (scipy.ndimage.label with 4-connectivity, size filter,
                  raster numbering)
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None

DTYPES = {'u16': 0, 'f16': 1, 'f32': 2}


class OrPlane(ctypes.Structure):
    _fields_ = [('n', ctypes.c_double * 3), ('d', ctypes.c_double),
                ('n_inliers', ctypes.c_int), ('n_refit', ctypes.c_int),
                ('rms', ctypes.c_double), ('hyp_index', ctypes.c_int), ('band', ctypes.c_int)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        L.or_half_to_double.argtypes = [ctypes.c_uint16]
        L.or_half_to_double.restype = ctypes.c_double
        L.or_decode.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_long,
                                ctypes.c_double, P]
        L.or_decode.restype = ctypes.c_int
        L.or_diffuse.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int]
        L.or_diffuse.restype = ctypes.c_int
        L.or_normals.argtypes = [P, ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 + \
            [ctypes.c_int, P, P, P]
        L.or_normals.restype = ctypes.c_int
        L.or_philox4x64.argtypes = [P, P, ctypes.c_int] + [ctypes.c_uint64] * 4 + [P]
        L.or_philox4x64.restype = None
        L.or_philox4x64_10.argtypes = [P, P, P]
        L.or_philox4x64_10.restype = None
        L.or_eig3.argtypes = [P, P, P]
        L.or_eig3.restype = None
        L.or_ransac.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_double,
                                ctypes.c_uint64, P, P, P]
        L.or_ransac.restype = ctypes.c_int
        L.or_ransac_regions.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_float, ctypes.c_uint64,
                                        ctypes.c_uint64, P]
        L.or_ransac_regions.restype = ctypes.c_int
        L.or_region_samples.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                        ctypes.c_uint64, P]
        L.or_region_samples.restype = ctypes.c_int
        L.or_canny.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P]
        L.or_canny_sector.argtypes = [ctypes.c_int, ctypes.c_int]
        L.or_canny_sector.restype = ctypes.c_int
        L.or_canny.restype = ctypes.c_long
        L.or_segment.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
        L.or_segment.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


# ---------------------------------------------------------------------------
# stages
# ---------------------------------------------------------------------------

def decode(encoded: np.ndarray, dtype: str, depth_scale: float = 0.001) -> np.ndarray:
    """Sensor depth -> metres (float64), holes (0, <= 0, non-finite) -> 0."""
    e = np.ascontiguousarray(encoded)
    h, w = e.shape
    out = np.empty((h, w), dtype=np.float64)
    rc = lib().or_decode(_p(e), DTYPES[dtype], w, h, e.strides[0], depth_scale, _p(out))
    if rc != 0:
        raise ValueError('or_decode failed')
    return out


def diffuse(depth: np.ndarray, iters: int, lam: float = 0.2, K: float = 0.02,
            mode: int = 0) -> np.ndarray:
    """Eq. 1 / Alg. 1 Jacobi diffusion in FP64 (mode 0 = PM4, 1 = ALG1)."""
    z = np.ascontiguousarray(depth, dtype=np.float64)
    h, w = z.shape
    out = np.empty_like(z)
    rc = lib().or_diffuse(_p(z), _p(out), w, h, iters, lam, K, mode)
    if rc != 0:
        raise ValueError('or_diffuse failed (%d)' % rc)
    return out


def normals(depth: np.ndarray, intr, stencil: int = 0):
    """Back-projected points, unit normals (SoA [3][h][w]) and validity bits."""
    z = np.ascontiguousarray(depth, dtype=np.float64)
    h, w = z.shape
    P = np.empty((3, h, w), dtype=np.float64)
    N = np.empty((3, h, w), dtype=np.float64)
    V = np.empty((h, w), dtype=np.uint8)
    fx, fy, cx, cy = intr
    rc = lib().or_normals(_p(z), w, h, fx, fy, cx, cy, stencil, _p(P), _p(N), _p(V))
    if rc != 0:
        raise ValueError('or_normals failed')
    return P, N, V


PHILOX_M = (0xD2E7470EE14C6C93, 0xCA5A826395121157)
PHILOX_W = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)


def philox4x64(ctr, key, rounds=10, m=PHILOX_M, wc=PHILOX_W):
    c = np.asarray(ctr, dtype=np.uint64)
    k = np.asarray(key, dtype=np.uint64)
    out = np.empty(4, dtype=np.uint64)
    lib().or_philox4x64(_p(c), _p(k), rounds, m[0], m[1], wc[0], wc[1], _p(out))
    return out


def philox4x64_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint64)
    k = np.asarray(key, dtype=np.uint64)
    out = np.empty(4, dtype=np.uint64)
    lib().or_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def eig3(A: np.ndarray):
    a = np.ascontiguousarray(A, dtype=np.float64).reshape(9)
    ev = np.empty(3)
    V = np.empty(9)
    lib().or_eig3(_p(a), _p(ev), _p(V))
    return ev, V.reshape(3, 3)


@dataclass
class RansacResult:
    planes: np.ndarray        # (n, 4) n_x, n_y, n_z, d
    n_inliers: np.ndarray
    n_refit: np.ndarray
    rms: np.ndarray
    hyp_index: np.ndarray
    band: np.ndarray          # near-threshold candidates per plane (FP64 residual within 1e-6 m)
    labels: np.ndarray        # (h, w) int16, -1 = none
    counts: np.ndarray        # (max_planes, H) per-round hypothesis counts (rounds not run: 0)


def ransac(P32: np.ndarray, N32, valid: np.ndarray, hypotheses: int, thr: float,
           max_planes: int, min_inliers: int, seed: int, gate_deg: float = 20.0,
           frame_idx: int = 0) -> RansacResult:
    """Sequential multi-plane RANSAC (Alg. 2, whole frame) on FP32 points."""
    P = np.ascontiguousarray(P32, dtype=np.float32)
    _, h, w = P.shape
    N = None if N32 is None else np.ascontiguousarray(N32, dtype=np.float32)
    V = np.ascontiguousarray(valid, dtype=np.uint8)
    planes = (OrPlane * max_planes)()
    labels = np.empty((h, w), dtype=np.int16)
    counts = np.zeros((max_planes, hypotheses), dtype=np.int32)
    n = lib().or_ransac(_p(P), _p(N), _p(V), w, h, hypotheses, thr, max_planes, min_inliers,
                        seed, gate_deg, frame_idx, ctypes.cast(planes, ctypes.c_void_p),
                        _p(labels), _p(counts))
    if n < 0:
        raise ValueError('or_ransac failed (%d)' % n)
    pl = np.array([[*planes[i].n, planes[i].d] for i in range(n)]).reshape(-1, 4)
    f = lambda k: np.array([getattr(planes[i], k) for i in range(n)])
    return RansacResult(pl, f('n_inliers'), f('n_refit'), f('rms'), f('hyp_index'), f('band'),
                        labels, counts)


class OrRegionPlane(ctypes.Structure):
    _fields_ = [('n', ctypes.c_double * 3), ('d', ctypes.c_double),
                ('error', ctypes.c_ulonglong), ('inliers', ctypes.c_int),
                ('total', ctypes.c_int), ('accepted', ctypes.c_int), ('hyp_index', ctypes.c_int)]


REGION_ERROR_UNIT = 2.0 ** -32      # metres per unit of the integer distance sums


@dataclass
class RegionResult:
    planes: np.ndarray        # (R, 4) winning hypothesis planes (FP32 values), 0 if none
    error: np.ndarray         # (R,) uint64 sum of distances in units of 2^-32 m
    inliers: np.ndarray
    total: np.ndarray
    accepted: np.ndarray      # (R,) bool: inliers / total > 0.9
    hyp_index: np.ndarray     # (R,) -1 if the region had no usable hypothesis


def ransac_regions(P32: np.ndarray, valid: np.ndarray, regions: np.ndarray, n_regions: int,
                   hypotheses: int, thr: float, seed: int, frame_idx: int = 0) -> RegionResult:
    """Alg. 2 per region: minimum total distance, 0.9 inlier-ratio acceptance."""
    P = np.ascontiguousarray(P32, dtype=np.float32)
    _, h, w = P.shape
    V = np.ascontiguousarray(valid, dtype=np.uint8)
    Rg = np.ascontiguousarray(regions, dtype=np.int32)
    out = (OrRegionPlane * n_regions)()
    rc = lib().or_ransac_regions(_p(P), _p(V), _p(Rg), w, h, n_regions, hypotheses, thr, seed,
                                 frame_idx, ctypes.cast(out, ctypes.c_void_p))
    if rc < 0:
        raise ValueError('or_ransac_regions failed (%d)' % rc)
    g = lambda k, t: np.array([getattr(out[i], k) for i in range(n_regions)], dtype=t)
    pl = np.array([[*out[i].n, out[i].d] for i in range(n_regions)]).reshape(-1, 4)
    return RegionResult(pl, g('error', np.uint64), g('inliers', np.int64), g('total', np.int64),
                        g('accepted', np.int64).astype(bool), g('hyp_index', np.int64))


def region_samples(valid: np.ndarray, regions: np.ndarray, n_regions: int, r: int, hyp: int,
                   seed: int, frame_idx: int = 0):
    """Pixel indices of the three samples of hypothesis `hyp` of region r, or None."""
    V = np.ascontiguousarray(valid, dtype=np.uint8)
    Rg = np.ascontiguousarray(regions, dtype=np.int32)
    h, w = Rg.shape
    out = np.zeros(3, dtype=np.int64)
    ok = lib().or_region_samples(_p(Rg), _p(V), w, h, n_regions, r, hyp, seed, frame_idx,
                                 _p(out))
    return out if ok else None


def canny(N32: np.ndarray, valid: np.ndarray, low: int = 60, high: int = 150,
          states: bool = False):
    """Canny edges of the 8-bit normal image (Sec. III-D); u8 [h, w], 1 = edge.
    states=True also returns the pre-hysteresis state image (0/1/2)."""
    N = np.ascontiguousarray(N32, dtype=np.float32)
    _, h, w = N.shape
    V = np.ascontiguousarray(valid, dtype=np.uint8)
    out = np.zeros((h, w), dtype=np.uint8)
    st = np.zeros((h, w), dtype=np.uint8) if states else None
    rc = lib().or_canny(_p(N), _p(V), w, h, low, high, _p(out), _p(st))
    if rc < 0:
        raise ValueError('or_canny failed (%d)' % rc)
    return (out, st) if states else out


def canny_sector(gx: int, gy: int) -> int:
    """The gradient direction sector of the non-maximum suppression."""
    return lib().or_canny_sector(int(gx), int(gy))


def segment(edges: np.ndarray, valid: np.ndarray, min_pixels: int = 200, gap: int = 1):
    """4-connected regions of valid pixels away from edges: (int32 labels [h, w], R)."""
    E = np.ascontiguousarray(edges, dtype=np.uint8)
    V = np.ascontiguousarray(valid, dtype=np.uint8)
    h, w = E.shape
    out = np.zeros((h, w), dtype=np.int32)
    R = lib().or_segment(_p(E), _p(V), w, h, gap, min_pixels, _p(out))
    if R < 0:
        raise ValueError('or_segment failed (%d)' % R)
    return out, R


# ---------------------------------------------------------------------------
# the whole per-frame path
# ---------------------------------------------------------------------------

@dataclass
class FrameResult:
    depth: np.ndarray         # diffused depth, FP64
    P: np.ndarray
    N: np.ndarray
    valid: np.ndarray
    ransac: RansacResult


def process_frame(encoded, dtype, intr, iters, lam=0.2, K=0.02, mode=0, stencil=0,
                  hypotheses=1024, thr=0.01, max_planes=12, min_inliers=100, seed=0,
                  gate_deg=20.0, frame_idx=0, depth_scale=0.001) -> FrameResult:
    """decode -> diffuse (FP64) -> normals (FP64) -> FP32 points -> RANSAC."""
    z = decode(encoded, dtype, depth_scale)
    zs = diffuse(z, iters, lam, K, mode)
    P, N, V = normals(zs, intr, stencil)
    r = ransac(P.astype(np.float32), N.astype(np.float32), V, hypotheses, thr, max_planes,
               min_inliers, seed, gate_deg, frame_idx)
    return FrameResult(zs, P, N, V, r)
