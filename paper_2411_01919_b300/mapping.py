"""Binding of the polygon map manager (Sec. III-E, Eq. 4-10; host code in
libpm, csrc/map.cpp), and the host step that turns the planar regions of a
frame into polygons (the convex hull of each region's points on its plane)."""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import _ffi
from ._ffi import check


@dataclass
class MapParams:
    drift_tolerance_m: float = 0.05            # Eq. 5
    sigma_p: float = 1e-5
    sigma_m: float = 1e-4
    initial_variance: float = 1e-4
    horizontal_cos: float = math.cos(math.radians(20.0))
    min_overlap_m2: float = 1e-4


class MapManager:
    """Integrates per-frame polygons (camera frame) with the odometry pose."""

    def __init__(self, params: Optional[MapParams] = None):
        self.lib = _ffi.load()
        self.p = params or MapParams()
        mp = _ffi.MapParams(self.p.drift_tolerance_m, self.p.sigma_p, self.p.sigma_m,
                            self.p.initial_variance, self.p.horizontal_cos, self.p.min_overlap_m2)
        h = ctypes.c_void_p()
        check(self.lib.pm_map_create(ctypes.byref(mp), ctypes.byref(h)))
        self._h = h

    def close(self):
        if self._h:
            self.lib.pm_map_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def integrate(self, pose: np.ndarray, polygons: Sequence[Tuple[np.ndarray, float, np.ndarray]]):
        """pose: 4x4 map <- camera; polygons: (n [3], d, vertices [k, 3]) in the camera frame."""
        pose = np.ascontiguousarray(pose, dtype=np.float64).reshape(16)
        keep = []
        arr = (_ffi.Polygon * max(1, len(polygons)))()
        for i, (n, d, V) in enumerate(polygons):
            V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1, 3)
            keep.append(V)
            arr[i].n = (ctypes.c_double * 3)(*[float(v) for v in n])
            arr[i].d = float(d)
            arr[i].vertices = V.ctypes.data_as(ctypes.c_void_p)
            arr[i].n_vertices = len(V)
        st = _ffi.MapStep()
        check(self.lib.pm_map_integrate(self._h, pose.ctypes.data_as(ctypes.c_void_p), arr,
                                        len(polygons), ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in _ffi.MapStep._fields_}

    def __len__(self):
        return int(self.lib.pm_map_size(self._h))

    def polygon(self, i: int):
        """(footprint [k, 2] counter-clockwise, height, area, observations)."""
        n = ctypes.c_int(0)
        check(self.lib.pm_map_polygon(self._h, i, None, None, None, None, 0, ctypes.byref(n)))
        xy = np.zeros((n.value, 2), dtype=np.float64)
        z, a, obs = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_int(0)
        check(self.lib.pm_map_polygon(self._h, i, ctypes.byref(z), ctypes.byref(a),
                                      ctypes.byref(obs), xy.ctypes.data_as(ctypes.c_void_p),
                                      n.value, ctypes.byref(n)))
        return xy, z.value, a.value, obs.value

    def polygons(self) -> List[tuple]:
        return [self.polygon(i) for i in range(len(self))]

    def drift(self) -> Tuple[float, float]:
        x, P = ctypes.c_double(0), ctypes.c_double(0)
        check(self.lib.pm_map_drift(self._h, ctypes.byref(x), ctypes.byref(P)))
        return x.value, P.value


def region_polygons(P: np.ndarray, labels: np.ndarray, planes: np.ndarray,
                    accepted: np.ndarray, min_points: int = 50):
    """Polygons of the accepted regions of one frame: each region's points are
    projected onto its plane and outlined by their convex hull there.
    P: [3, h, w] points, labels: [h, w] region ids, planes: [R, 4] (n, d)."""
    pts = P.reshape(3, -1).T.astype(np.float64)
    lab = labels.reshape(-1)
    out = []
    for r in range(len(planes)):
        if not accepted[r]:
            continue
        X = pts[lab == r]
        if len(X) < min_points:
            continue
        n = planes[r, :3] / np.linalg.norm(planes[r, :3])
        d = planes[r, 3] / np.linalg.norm(planes[r, :3])
        Xp = X - np.outer(X @ n + d, n)
        e1 = np.cross(n, [1.0, 0.0, 0.0] if abs(n[0]) < 0.9 else [0.0, 1.0, 0.0])
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(n, e1)
        uv = np.stack([Xp @ e1, Xp @ e2], axis=1)
        idx = _hull_indices(uv)
        if len(idx) >= 3:
            out.append((n, float(d), Xp[idx]))
    return out


def _hull_indices(uv: np.ndarray) -> List[int]:
    order = np.lexsort((uv[:, 1], uv[:, 0]))
    cr = lambda o, a, b: (uv[a, 0] - uv[o, 0]) * (uv[b, 1] - uv[o, 1]) - \
        (uv[a, 1] - uv[o, 1]) * (uv[b, 0] - uv[o, 0])
    lower, upper = [], []
    for i in order:
        while len(lower) >= 2 and cr(lower[-2], lower[-1], i) <= 0:
            lower.pop()
        lower.append(i)
    for i in order[::-1]:
        while len(upper) >= 2 and cr(upper[-2], upper[-1], i) <= 0:
            upper.pop()
        upper.append(i)
    return lower[:-1] + upper[:-1]
