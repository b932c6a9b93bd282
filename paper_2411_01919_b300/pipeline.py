"""Python binding of libpm: the depth -> diffusion -> normals -> planes path.

Thin layer over the C ABI: it checks tensor placement and dtypes, passes raw
device pointers and the current CUDA stream, and wraps results.  Every step
of the path runs in libpm's CUDA kernels; there is no CPU or PyTorch fallback.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _ffi
from ._ffi import check

_DT = {torch.uint16: _ffi.PM_U16_MM, torch.float16: _ffi.PM_F16_M, torch.float32: _ffi.PM_F32_M}
_NP_DT = {np.dtype(np.uint16): _ffi.PM_U16_MM, np.dtype(np.float16): _ffi.PM_F16_M,
          np.dtype(np.float32): _ffi.PM_F32_M}


@dataclass
class Params:
    """Parameters of the path (Alg. 1 and Alg. 2; see include/pm.h)."""
    iters: int = 30
    lam: float = 0.2
    K: float = 0.02
    mode: int = 0                 # 0 PM4, 1 ALG1
    iters_per_launch: int = 0     # temporal blocking depth, 0 = auto
    tile_w: int = 0               # fused-diffusion output tile, 0 = auto
    tile_h: int = 0
    hypotheses: int = 1024
    thr: float = 0.01
    max_planes: int = 12
    min_inliers: int = 100
    seed: int = 0
    gate_deg: float = 20.0
    stencil: int = 0              # 0 central, 1 Sobel
    depth_scale: float = 0.001


# pm_plane as a numpy record (include/pm.h): the planes array a call fills is
# read as one structured view instead of field by field
_PLANE_DT = np.dtype([('n', '<f8', (3,)), ('d', '<f8'), ('n_inliers', '<i4'),
                      ('n_refit', '<i4'), ('rms', '<f4'), ('hyp_index', '<i4')])
assert _PLANE_DT.itemsize == ctypes.sizeof(_ffi.Plane)


@dataclass
class Planes:
    """Planes of one frame: rows (nx, ny, nz, d) with n . X + d = 0."""
    planes: np.ndarray
    n_inliers: np.ndarray
    n_refit: np.ndarray
    rms: np.ndarray
    hyp_index: np.ndarray
    labels: Optional[torch.Tensor] = None

    @staticmethod
    def from_c(arr, n, labels=None) -> 'Planes':
        a = np.frombuffer(arr, dtype=_PLANE_DT, count=n)
        pl = np.concatenate([a['n'], a['d'][:, None]], axis=1)
        return Planes(pl, a['n_inliers'].astype(np.int64), a['n_refit'].astype(np.int64),
                      a['rms'].astype(np.float64), a['hyp_index'].astype(np.int64), labels)


@dataclass
class RegionPlanes:
    """One model per region (Alg. 2 per polygon): rows (nx, ny, nz, d) of the
    winning hypothesis, its distance sum (units of 2^-32 m), inlier and point
    counts, the 90% acceptance flag and the hypothesis index (-1: none)."""
    planes: np.ndarray
    error: np.ndarray
    inliers: np.ndarray
    total: np.ndarray
    accepted: np.ndarray
    hyp_index: np.ndarray

    @staticmethod
    def from_c(arr, n) -> 'RegionPlanes':
        pl = np.array([[*arr[i].n, arr[i].d] for i in range(n)], dtype=np.float64).reshape(-1, 4)
        g = lambda k, t: np.array([getattr(arr[i], k) for i in range(n)], dtype=t)
        return RegionPlanes(pl, g('error', np.uint64), g('inliers', np.int64), g('total', np.int64),
                            g('accepted', np.int64).astype(bool), g('hyp_index', np.int64))


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, what: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError('%s must be a CUDA tensor' % what)
    return ctypes.c_void_p(t.data_ptr())


def _intr(K) -> _ffi.Intrinsics:
    fx, fy, cx, cy = (float(x) for x in K)
    return _ffi.Intrinsics(fx, fy, cx, cy)


def _depth_args(depth: torch.Tensor):
    if depth.dim() != 2:
        raise ValueError('depth must be a 2-D [h, w] tensor')
    if depth.dtype not in _DT:
        raise ValueError('depth dtype must be uint16 (mm), float16 or float32 (m)')
    if depth.stride(1) != 1:
        raise ValueError('depth rows must be contiguous')
    h, w = depth.shape
    pitch = depth.stride(0) * depth.element_size()
    return _DT[depth.dtype], w, h, pitch


class Pipeline:
    """A libpm context: device scratch for `max_frames` frames of up to
    max_w x max_h pixels on the current CUDA device."""

    def __init__(self, params: Params = None, max_w: int = 640, max_h: int = 480,
                 max_frames: int = 1, lib_path: str = None):
        # a copy: set_tiling changes this context's parameters, never those of
        # another context built from the same Params
        self.p = replace(params) if params is not None else Params()
        self.lib = _ffi.load(lib_path) if lib_path else _ffi.load()
        p = self.p
        self._dp = _ffi.DiffusionParams(p.iters, p.lam, p.K, p.mode, p.iters_per_launch,
                                        p.tile_w, p.tile_h)
        self._rp = _ffi.RansacParams(p.hypotheses, p.thr, p.max_planes, p.min_inliers,
                                     p.seed, p.gate_deg)
        self._mp = _ffi.MiscParams(p.stencil, p.depth_scale)
        self.max_w, self.max_h, self.max_frames = max_w, max_h, max_frames
        h = ctypes.c_void_p()
        check(self.lib.pm_create(ctypes.byref(self._dp), ctypes.byref(self._rp),
                                 ctypes.byref(self._mp), max_w, max_h, max_frames,
                                 ctypes.byref(h)))
        self._h = h
        self._pending = 0

    def close(self):
        if getattr(self, '_h', None):
            self.lib.pm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- stages -------------------------------------------------------------
    def diffuse(self, depth: torch.Tensor, out: torch.Tensor = None, stream=None) -> torch.Tensor:
        dt, w, h, pitch = _depth_args(depth)
        if out is None:
            out = torch.empty((h, w), dtype=torch.float32, device=depth.device)
        if out.dtype != torch.float32 or not out.is_contiguous() or tuple(out.shape) != (h, w):
            raise ValueError('out must be a contiguous float32 [h, w] tensor')
        check(self.lib.pm_diffuse(self._h, _dev(depth, 'depth'), dt, w, h, pitch,
                                  _dev(out, 'out'), _stream_ptr(stream)))
        return out

    def normals(self, depth: torch.Tensor, K, stream=None, out=None):
        """Points, normals and validity of an FP32 depth image; `out` = (P, N, V)
        to write into given tensors (float32 [3, h, w] twice, uint8 [h, w])."""
        if depth.dtype != torch.float32 or not depth.is_contiguous() or depth.dim() != 2:
            raise ValueError('depth must be a contiguous float32 [h, w] tensor')
        h, w = depth.shape
        if out is not None:
            P, N, V = out
            for t, shape, dt in ((P, (3, h, w), torch.float32), (N, (3, h, w), torch.float32),
                                 (V, (h, w), torch.uint8)):
                if tuple(t.shape) != shape or t.dtype != dt or not t.is_contiguous():
                    raise ValueError('out tensors must be contiguous float32 [3, h, w] x 2 '
                                     'and uint8 [h, w]')
        else:
            P = torch.empty((3, h, w), dtype=torch.float32, device=depth.device)
            N = torch.empty((3, h, w), dtype=torch.float32, device=depth.device)
            V = torch.empty((h, w), dtype=torch.uint8, device=depth.device)
        k = _intr(K)
        check(self.lib.pm_normals(self._h, _dev(depth, 'depth'), w, h, ctypes.byref(k),
                                  _dev(P, 'P'), _dev(N, 'N'), _dev(V, 'V'), _stream_ptr(stream)))
        return P, N, V

    def ransac_planes(self, P: torch.Tensor, N: Optional[torch.Tensor], valid: torch.Tensor,
                      frame_idx: int = 0, labels: bool = True, stream=None) -> Planes:
        _, h, w = P.shape
        for t, nm in ((P, 'P'), (valid, 'valid')):
            if not t.is_contiguous():
                raise ValueError('%s must be contiguous' % nm)
        if P.dtype != torch.float32 or valid.dtype != torch.uint8:
            raise ValueError('P must be float32 and valid uint8')
        lab = torch.empty((h, w), dtype=torch.int16, device=P.device) if labels else None
        arr = (_ffi.Plane * self.p.max_planes)()
        n = ctypes.c_int(0)
        check(self.lib.pm_ransac_planes(
            self._h, _dev(P, 'P'), _dev(N, 'N') if N is not None else None, _dev(valid, 'valid'),
            w, h, frame_idx, arr, self.p.max_planes, ctypes.byref(n),
            _dev(lab, 'labels') if lab is not None else None, _stream_ptr(stream)))
        return Planes.from_c(arr, n.value, lab)

    def ransac_regions(self, P: torch.Tensor, valid: torch.Tensor, regions: torch.Tensor,
                       n_regions: int, hypotheses: int = 256, frame_idx: int = 0,
                       stream=None) -> RegionPlanes:
        """Per-region RANSAC (Alg. 2 per polygon); regions: int32 [h, w], -1 = none."""
        _, h, w = P.shape
        for t, nm in ((P, 'P'), (valid, 'valid'), (regions, 'regions')):
            if not t.is_contiguous():
                raise ValueError('%s must be contiguous' % nm)
        if P.dtype != torch.float32 or valid.dtype != torch.uint8 or regions.dtype != torch.int32:
            raise ValueError('P must be float32, valid uint8 and regions int32')
        if tuple(valid.shape) != (h, w) or tuple(regions.shape) != (h, w):
            raise ValueError('valid and regions must be [h, w] like P')
        arr = (_ffi.RegionPlane * max(n_regions, 1))()
        check(self.lib.pm_ransac_regions(
            self._h, _dev(P, 'P'), _dev(valid, 'valid'), _dev(regions, 'regions'), w, h, n_regions,
            hypotheses, frame_idx, arr, _stream_ptr(stream)))
        return RegionPlanes.from_c(arr, n_regions)

    def canny(self, N: torch.Tensor, valid: torch.Tensor, low: int = 60, high: int = 150,
              stream=None) -> torch.Tensor:
        """Canny edges of the normal image (Sec. III-D): u8 [h, w], 1 = edge."""
        _, h, w = N.shape
        if N.dtype != torch.float32 or valid.dtype != torch.uint8 or not N.is_contiguous() \
                or not valid.is_contiguous() or tuple(valid.shape) != (h, w):
            raise ValueError('N must be contiguous float32 [3, h, w] and valid uint8 [h, w]')
        E = torch.empty((h, w), dtype=torch.uint8, device=N.device)
        check(self.lib.pm_canny(self._h, _dev(N, 'N'), _dev(valid, 'valid'), w, h, low, high,
                                _dev(E, 'edges'), _stream_ptr(stream)))
        return E

    def segment(self, edges: torch.Tensor, valid: torch.Tensor, min_pixels: int = 200,
                gap: int = 1, stream=None):
        """Regions bounded by the edges: (int32 labels [h, w], number of regions)."""
        h, w = edges.shape
        if edges.dtype != torch.uint8 or valid.dtype != torch.uint8 or not edges.is_contiguous() \
                or not valid.is_contiguous() or tuple(valid.shape) != (h, w):
            raise ValueError('edges and valid must be contiguous uint8 [h, w]')
        lab = torch.empty((h, w), dtype=torch.int32, device=edges.device)
        n = ctypes.c_int(0)
        check(self.lib.pm_segment(self._h, _dev(edges, 'edges'), _dev(valid, 'valid'), w, h, gap,
                                  min_pixels, _dev(lab, 'labels'), ctypes.byref(n),
                                  _stream_ptr(stream)))
        return lab, n.value

    # -- whole path ---------------------------------------------------------
    def process_frame(self, depth: torch.Tensor, K, frame_idx: int = 0, labels: bool = True,
                      stream=None) -> Planes:
        dt, w, h, pitch = _depth_args(depth)
        lab = torch.empty((h, w), dtype=torch.int16, device=depth.device) if labels else None
        arr = (_ffi.Plane * self.p.max_planes)()
        n = ctypes.c_int(0)
        k = _intr(K)
        check(self.lib.pm_process_frame(
            self._h, _dev(depth, 'depth'), dt, w, h, pitch, ctypes.byref(k), frame_idx, arr,
            self.p.max_planes, ctypes.byref(n), _dev(lab, 'labels') if lab is not None else None,
            _stream_ptr(stream)))
        return Planes.from_c(arr, n.value, lab)

    def process_frame_host(self, depth: np.ndarray, K, frame_idx: int = 0,
                           labels: Optional[np.ndarray] = None, stream=None) -> Planes:
        """Host depth in, host planes (and optionally host labels) out."""
        if depth.ndim != 2 or depth.dtype not in _NP_DT:
            raise ValueError('depth must be a 2-D uint16/float16/float32 array')
        h, w = depth.shape
        if depth.strides[1] != depth.itemsize:
            raise ValueError('depth rows must be contiguous')
        if labels is not None and (labels.dtype != np.int16 or labels.shape != (h, w)
                                   or not labels.flags.c_contiguous):
            raise ValueError('labels must be a contiguous int16 [h, w] array')
        arr = (_ffi.Plane * self.p.max_planes)()
        n = ctypes.c_int(0)
        k = _intr(K)
        check(self.lib.pm_process_frame_host(
            self._h, ctypes.c_void_p(depth.ctypes.data), _NP_DT[depth.dtype], w, h,
            depth.strides[0], ctypes.byref(k), frame_idx, arr, self.p.max_planes, ctypes.byref(n),
            ctypes.c_void_p(labels.ctypes.data) if labels is not None else None,
            _stream_ptr(stream)))
        return Planes.from_c(arr, n.value)

    # -- batched form -------------------------------------------------------
    def _frames(self, frames: Sequence[dict]):
        n = len(frames)
        arr = (_ffi.Frame * n)()
        for i, fr in enumerate(frames):
            dt, w, h, pitch = _depth_args(fr['depth'])
            lab = fr.get('labels')
            out = fr.get('depth_out')
            arr[i] = _ffi.Frame(ctypes.c_void_p(fr['depth'].data_ptr()), dt, w, h, pitch,
                                _intr(fr['K']), int(fr.get('frame_idx', 0)),
                                int(fr.get('iters', -1)),
                                ctypes.c_void_p(lab.data_ptr()) if lab is not None else None,
                                ctypes.c_void_p(out.data_ptr()) if out is not None else None)
        return arr

    def process_batch(self, frames: Sequence[dict], use_graph: bool = True,
                      stream=None) -> List[Planes]:
        """frames: dicts with 'depth' (CUDA [h, w] tensor), 'K', optional
        'frame_idx', 'iters', 'labels' (int16 CUDA [h, w]) and 'depth_out'."""
        n = len(frames)
        arr = self._frames(frames)
        mp = self.p.max_planes
        planes = (_ffi.Plane * (n * mp))()
        counts = (ctypes.c_int * n)()
        check(self.lib.pm_process_batch(self._h, arr, n, planes, counts, int(use_graph),
                                        _stream_ptr(stream)))
        out = []
        for i in range(n):
            sub = (_ffi.Plane * mp).from_address(ctypes.addressof(planes) + i * mp *
                                                 ctypes.sizeof(_ffi.Plane))
            out.append(Planes.from_c(sub, counts[i], frames[i].get('labels')))
        return out

    def submit_batch(self, frames: Sequence[dict], use_graph: bool = True, stream=None):
        """Enqueue a batch and return at once; call collect_batch() after the
        stream has reached this point."""
        arr = self._frames(frames)
        check(self.lib.pm_process_batch_async(self._h, arr, len(frames), int(use_graph),
                                              _stream_ptr(stream)))
        self._pending = len(frames)
        self._pending_frames = list(frames)

    def submit_batch_host(self, frames: Sequence[dict], use_graph: bool = True, stream=None):
        """As submit_batch, with each frame's 'depth' a CPU tensor or numpy array
        (pinned memory for asynchronous copies) that the call copies to the
        device itself; it must stay unchanged until collect_batch()."""
        n = len(frames)
        arr = (_ffi.Frame * n)()
        keep = []
        for i, fr in enumerate(frames):
            d = fr['depth']
            if isinstance(d, torch.Tensor):
                if d.is_cuda or d.dim() != 2 or d.dtype not in _DT or d.stride(1) != 1:
                    raise ValueError('depth must be a 2-D host tensor with contiguous rows')
                dt, ptr = _DT[d.dtype], d.data_ptr()
                pitch = d.stride(0) * d.element_size()
            else:
                if d.ndim != 2 or d.dtype not in _NP_DT or d.strides[1] != d.itemsize:
                    raise ValueError('depth must be a 2-D uint16/float16/float32 array')
                dt, ptr, pitch = _NP_DT[d.dtype], d.ctypes.data, d.strides[0]
            keep.append(d)
            h, w = d.shape
            lab = fr.get('labels')
            out = fr.get('depth_out')
            arr[i] = _ffi.Frame(ctypes.c_void_p(ptr), dt, w, h, pitch, _intr(fr['K']),
                                int(fr.get('frame_idx', 0)), int(fr.get('iters', -1)),
                                ctypes.c_void_p(lab.data_ptr()) if lab is not None else None,
                                ctypes.c_void_p(out.data_ptr()) if out is not None else None)
        check(self.lib.pm_process_batch_host_async(self._h, arr, n, int(use_graph),
                                                   _stream_ptr(stream)))
        self._pending = n
        self._pending_frames = list(frames)
        self._host_keep = keep

    def collect_batch(self) -> List[Planes]:
        n = self._pending
        mp = self.p.max_planes
        planes = (_ffi.Plane * (max(n, 1) * mp))()
        counts = (ctypes.c_int * max(n, 1))()
        check(self.lib.pm_batch_collect(self._h, planes, counts, n))
        self._pending = 0
        out = []
        for i in range(n):
            sub = (_ffi.Plane * mp).from_address(ctypes.addressof(planes) + i * mp *
                                                 ctypes.sizeof(_ffi.Plane))
            out.append(Planes.from_c(sub, counts[i], self._pending_frames[i].get('labels')))
        return out

    def frame_geometry(self, frame: int, w: int, h: int, device=None, stream=None):
        """Points, normals (float32 [3, h, w]) and validity (uint8 [h, w]) that
        the RANSAC stage of the last whole-path call used for batch frame
        `frame` (of size w x h)."""
        dev = device if device is not None else torch.device('cuda', torch.cuda.current_device())
        P = torch.empty((3, h, w), dtype=torch.float32, device=dev)
        N = torch.empty((3, h, w), dtype=torch.float32, device=dev)
        V = torch.empty((h, w), dtype=torch.uint8, device=dev)
        check(self.lib.pm_frame_geometry(self._h, int(frame), _dev(P, 'P'), _dev(N, 'N'),
                                         _dev(V, 'V'), _stream_ptr(stream)))
        return P, N, V

    def set_tiling(self, iters_per_launch: int = 0, tile_w: int = 0, tile_h: int = 0):
        """Diffusion tiling (bit-identical results for every choice)."""
        check(self.lib.pm_set_tiling(self._h, iters_per_launch, tile_w, tile_h))
        self.p.iters_per_launch, self.p.tile_w, self.p.tile_h = iters_per_launch, tile_w, tile_h

    # -- instrumentation ----------------------------------------------------
    def set_timing(self, mode: int = 1):
        """0 off, 1 per-stage events, 2 events around every scoring launch."""
        check(self.lib.pm_set_timing(self._h, int(mode)))

    def kernel_stats(self):
        ms = ctypes.c_float(0)
        pairs = ctypes.c_longlong(0)
        evaluated = ctypes.c_longlong(0)
        nl = ctypes.c_int(0)
        launches = ctypes.c_longlong(0)
        check(self.lib.pm_kernel_stats(self._h, ctypes.byref(ms), ctypes.byref(pairs),
                                       ctypes.byref(evaluated), ctypes.byref(nl),
                                       ctypes.byref(launches)))
        return {'score_ms': ms.value, 'score_pairs': pairs.value,
                'evaluated_pairs': evaluated.value, 'score_launches': nl.value,
                'launches': launches.value}

    def stage_times(self):
        ms = (ctypes.c_float * 3)()
        check(self.lib.pm_stage_times(self._h, ms))
        return {'diffuse_ms': ms[0], 'normals_ms': ms[1], 'ransac_ms': ms[2]}


def measure_peaks(stream=None) -> dict:
    """Measured FP32 FMA (TFLOP/s) and ex2 (Top/s) throughput of the current
    device, and its SM count (pm_measure_peaks)."""
    f, x, n = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_int(0)
    check(_ffi.load().pm_measure_peaks(ctypes.byref(f), ctypes.byref(x), ctypes.byref(n),
                                       _stream_ptr(stream)))
    return {'fp32_tflops': f.value, 'ex2_tops': x.value, 'sm_count': n.value}


def scratch_bytes(max_w, max_h, max_frames, hypotheses, max_planes) -> int:
    return int(_ffi.load().pm_scratch_bytes(max_w, max_h, max_frames, hypotheses, max_planes))
