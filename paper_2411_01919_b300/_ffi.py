"""ctypes declarations of libpm's C ABI (include/pm.h).  Marshalling only."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, 'libpm.so')

PM_OK, PM_ERR_ARG, PM_ERR_OOM, PM_ERR_CUDA, PM_ERR_TIMEOUT, PM_ERR_STATE = range(6)
STATUS = {0: 'PM_OK', 1: 'PM_ERR_ARG', 2: 'PM_ERR_OOM', 3: 'PM_ERR_CUDA', 4: 'PM_ERR_TIMEOUT',
          5: 'PM_ERR_STATE'}
PM_U16_MM, PM_F16_M, PM_F32_M = 0, 1, 2
PM_NOALLOC_MAX_PIXELS = 1 << 20


class Intrinsics(ctypes.Structure):
    _fields_ = [('fx', ctypes.c_double), ('fy', ctypes.c_double),
                ('cx', ctypes.c_double), ('cy', ctypes.c_double)]


class DiffusionParams(ctypes.Structure):
    _fields_ = [('iters', ctypes.c_int), ('lambda_', ctypes.c_float), ('K', ctypes.c_float),
                ('mode', ctypes.c_int), ('iters_per_launch', ctypes.c_int),
                ('tile_w', ctypes.c_int), ('tile_h', ctypes.c_int)]


class RansacParams(ctypes.Structure):
    _fields_ = [('hypotheses', ctypes.c_int), ('thr_m', ctypes.c_float),
                ('max_planes', ctypes.c_int), ('min_inliers', ctypes.c_int),
                ('seed', ctypes.c_ulonglong), ('refit_normal_gate_deg', ctypes.c_float)]


class MiscParams(ctypes.Structure):
    _fields_ = [('normal_stencil', ctypes.c_int), ('depth_scale', ctypes.c_float)]


class Plane(ctypes.Structure):
    _fields_ = [('n', ctypes.c_double * 3), ('d', ctypes.c_double),
                ('n_inliers', ctypes.c_int), ('n_refit', ctypes.c_int),
                ('rms', ctypes.c_float), ('hyp_index', ctypes.c_int)]


class RegionPlane(ctypes.Structure):
    _fields_ = [('n', ctypes.c_double * 3), ('d', ctypes.c_double),
                ('error', ctypes.c_ulonglong), ('inliers', ctypes.c_int),
                ('total', ctypes.c_int), ('accepted', ctypes.c_int), ('hyp_index', ctypes.c_int)]


class MapParams(ctypes.Structure):
    _fields_ = [('drift_tolerance_m', ctypes.c_double), ('sigma_p', ctypes.c_double),
                ('sigma_m', ctypes.c_double), ('initial_variance', ctypes.c_double),
                ('horizontal_cos', ctypes.c_double), ('min_overlap_m2', ctypes.c_double)]


class Polygon(ctypes.Structure):
    _fields_ = [('n', ctypes.c_double * 3), ('d', ctypes.c_double),
                ('vertices', ctypes.c_void_p), ('n_vertices', ctypes.c_int)]


class MapStep(ctypes.Structure):
    _fields_ = [('matched', ctypes.c_int), ('merged', ctypes.c_int), ('added', ctypes.c_int),
                ('skipped', ctypes.c_int), ('measurement', ctypes.c_double),
                ('gain', ctypes.c_double), ('drift_prior', ctypes.c_double),
                ('drift', ctypes.c_double), ('variance', ctypes.c_double)]


class Frame(ctypes.Structure):
    _fields_ = [('depth', ctypes.c_void_p), ('dtype', ctypes.c_int), ('w', ctypes.c_int),
                ('h', ctypes.c_int), ('pitch', ctypes.c_int), ('K', Intrinsics),
                ('frame_idx', ctypes.c_ulonglong), ('iters', ctypes.c_int),
                ('labels', ctypes.c_void_p), ('depth_out', ctypes.c_void_p)]


EXPORTS = ['pm_create', 'pm_destroy', 'pm_diffuse', 'pm_normals', 'pm_ransac_planes',
           'pm_process_frame', 'pm_process_frame_host', 'pm_process_batch',
           'pm_process_batch_async', 'pm_process_batch_host_async', 'pm_batch_collect',
           'pm_frame_geometry',
           'pm_scratch_bytes', 'pm_set_timing',
           'pm_stage_times', 'pm_kernel_stats', 'pm_ransac_regions', 'pm_canny', 'pm_segment',
           'pm_map_create', 'pm_map_destroy', 'pm_map_integrate', 'pm_map_size',
           'pm_map_polygon', 'pm_map_drift', 'pm_diffuse_noalloc', 'pm_measure_peaks',
           'pm_set_tiling', 'pm_debug_bounds', 'pm_last_error']

_libs = {}


class PmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__('%s: %s' % (STATUS.get(status, status), msg))
        self.status = status


def load(path: str = LIB_PATH):
    """Load libpm.so (or another build of it, e.g. the bounds-checking one).
    Raises if the library is missing: there is no fallback."""
    if path in _libs:
        return _libs[path]
    if not os.path.exists(path):
        raise ImportError('libpm.so not found at %s; build it with '
                          '`python -m paper_2411_01919_b300.build`' % path)
    L = ctypes.CDLL(path)
    vp, i, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_ulonglong
    P = ctypes.POINTER
    sigs = {
        'pm_create': ([P(DiffusionParams), P(RansacParams), P(MiscParams), i, i, i, P(vp)], i),
        'pm_destroy': ([vp], None),
        'pm_diffuse': ([vp, vp, i, i, i, i, vp, vp], i),
        'pm_normals': ([vp, vp, i, i, P(Intrinsics), vp, vp, vp, vp], i),
        'pm_ransac_planes': ([vp, vp, vp, vp, i, i, u64, P(Plane), i, P(i), vp, vp], i),
        'pm_process_frame': ([vp, vp, i, i, i, i, P(Intrinsics), u64, P(Plane), i, P(i), vp, vp], i),
        'pm_process_frame_host': ([vp, vp, i, i, i, i, P(Intrinsics), u64, P(Plane), i, P(i), vp,
                                   vp], i),
        'pm_process_batch': ([vp, P(Frame), i, P(Plane), P(i), i, vp], i),
        'pm_process_batch_async': ([vp, P(Frame), i, i, vp], i),
        'pm_process_batch_host_async': ([vp, P(Frame), i, i, vp], i),
        'pm_batch_collect': ([vp, P(Plane), P(i), i], i),
        'pm_frame_geometry': ([vp, i, vp, vp, vp, vp], i),
        'pm_scratch_bytes': ([i, i, i, i, i], ctypes.c_longlong),
        'pm_set_timing': ([vp, i], i),
        'pm_stage_times': ([vp, P(ctypes.c_float)], i),
        'pm_kernel_stats': ([vp, P(ctypes.c_float), P(ctypes.c_longlong), P(ctypes.c_longlong),
                             P(i), P(ctypes.c_longlong)], i),
        'pm_ransac_regions': ([vp, vp, vp, vp, i, i, i, i, u64, P(RegionPlane), vp], i),
        'pm_canny': ([vp, vp, vp, i, i, i, i, vp, vp], i),
        'pm_segment': ([vp, vp, vp, i, i, i, i, vp, P(i), vp], i),
        'pm_map_create': ([P(MapParams), P(vp)], i),
        'pm_map_destroy': ([vp], None),
        'pm_map_integrate': ([vp, vp, P(Polygon), i, P(MapStep)], i),
        'pm_map_size': ([vp], i),
        'pm_map_polygon': ([vp, i, P(ctypes.c_double), P(ctypes.c_double), P(i), vp, i, P(i)], i),
        'pm_map_drift': ([vp, P(ctypes.c_double), P(ctypes.c_double)], i),
        'pm_diffuse_noalloc': ([vp, i, i, i, i, P(DiffusionParams), ctypes.c_float, vp, vp], i),
        'pm_measure_peaks': ([P(ctypes.c_double), P(ctypes.c_double), P(i), vp], i),
        'pm_set_tiling': ([vp, i, i, i], i),
        'pm_debug_bounds': ([P(ctypes.c_ulonglong)], i),
        'pm_last_error': ([], ctypes.c_char_p),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _libs[path] = L
    return L


def check(status: int):
    if status != PM_OK:
        raise PmError(status, load().pm_last_error().decode(errors='replace'))
