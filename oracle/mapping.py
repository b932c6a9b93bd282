"""Oracle of the polygon map manager (Sec. III-E, Eq. 4-10).

TEST INFRASTRUCTURE ONLY: the test suite is its only caller.

Plain FP64 Python, step by step in the order the section describes:
footprints of horizontal polygons in the map frame (hulls by Qhull through
scipy), matching by footprint overlap and centroid height within the drift
tolerance (Eq. 4-5), one scalar Kalman step per frame on the mean height
offset of the matches (Eq. 6-10), then compensation and merge-or-add.

Parity status: pinned (Kalman steady state and convergence in closed form,
overlap areas of rectangles in closed form and of random convex polygons by
Monte Carlo, merge decisions at the tolerance boundary, drift recovery on a
synthetic walk).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np
from scipy.spatial import ConvexHull


def hull_ccw(pts: np.ndarray) -> np.ndarray:
    """Convex hull of 2-D points, counter-clockwise (Qhull)."""
    pts = np.unique(np.asarray(pts, dtype=np.float64), axis=0)
    if len(pts) < 3:
        return pts
    try:
        h = ConvexHull(pts)
    except Exception:            # all points on a line: no area
        return pts[:0]
    return pts[h.vertices]


def area(poly: np.ndarray) -> float:
    """Signed shoelace area (positive for counter-clockwise)."""
    if len(poly) < 3:
        return 0.0
    x, y = poly[:, 0], poly[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


def centroid(poly: np.ndarray) -> Tuple[float, float]:
    x, y = poly[:, 0], poly[:, 1]
    xn, yn = np.roll(x, -1), np.roll(y, -1)
    f = x * yn - xn * y
    a = area(poly)
    return float(np.sum((x + xn) * f) / (6 * a)), float(np.sum((y + yn) * f) / (6 * a))


def clip_area(a: np.ndarray, b: np.ndarray) -> float:
    """Area of the intersection of two convex counter-clockwise polygons:
    keep the part of `a` on the left of every edge of `b`."""
    if len(a) < 3 or len(b) < 3:
        return 0.0
    out = [tuple(p) for p in a]
    for e in range(len(b)):
        p0, p1 = b[e], b[(e + 1) % len(b)]
        side = lambda q: (p1[0] - p0[0]) * (q[1] - p0[1]) - (p1[1] - p0[1]) * (q[0] - p0[0])
        pts, out = out, []
        for i in range(len(pts)):
            q, r = pts[i], pts[(i + 1) % len(pts)]
            sq, sr = side(q), side(r)
            if sq >= 0:
                out.append(q)
            if (sq >= 0) != (sr >= 0):
                t = sq / (sq - sr)
                out.append((q[0] + t * (r[0] - q[0]), q[1] + t * (r[1] - q[1])))
        if not out:
            return 0.0
    return abs(area(np.array(out))) if len(out) >= 3 else 0.0


@dataclass
class MapPolygon:
    xy: np.ndarray
    z: float
    area: float
    observations: int = 1


@dataclass
class MapOracle:
    tol: float = 0.05
    sigma_p: float = 1e-5
    sigma_m: float = 1e-4
    P: float = 1e-4
    horizontal_cos: float = float(np.cos(np.radians(20.0)))
    min_overlap: float = 1e-4
    x: float = 0.0
    polys: List[MapPolygon] = field(default_factory=list)

    def integrate(self, pose: np.ndarray, polygons: Sequence[Tuple[np.ndarray, float, np.ndarray]]):
        """pose: 4x4 map <- camera; polygons: (n [3], d, vertices [k, 3]) in the camera frame."""
        R, t = pose[:3, :3], pose[:3, 3]
        cand, skipped = [], 0
        for n, d, V in polygons:
            nw = R @ np.asarray(n, dtype=np.float64)
            if not abs(nw[2]) / np.linalg.norm(nw) >= self.horizontal_cos:
                skipped += 1
                continue
            dw = d - nw @ t
            W = (R @ np.asarray(V, dtype=np.float64).T).T + t
            fp = hull_ccw(W[:, :2])
            a = area(fp) if len(fp) >= 3 else 0.0
            if not a > 0:
                skipped += 1
                continue
            cx, cy = centroid(fp)
            z = -(nw[0] * cx + nw[1] * cy + dw) / nw[2]
            cand.append(MapPolygon(fp, z, a))
        # Eq. 4-5 against the map, with the drift estimate of the last frame
        match = []
        for c in cand:
            best, j_best = None, -1
            for j, m in enumerate(self.polys):
                dz = abs(c.z - self.x - m.z)
                if dz <= self.tol and (best is None or dz < best) and \
                        clip_area(c.xy, m.xy) > self.min_overlap:
                    best, j_best = dz, j
            match.append(j_best)
        offsets = [c.z - self.polys[j].z for c, j in zip(cand, match) if j >= 0]
        # Eq. 6-10
        x_prior = self.x
        self.P = self.P + self.sigma_p
        K = zk = 0.0
        if offsets:
            zk = sum(offsets) / len(offsets)
            K = self.P / (self.P + self.sigma_m)
            self.x = self.x + K * (zk - self.x)
            self.P = (1 - K) * self.P
        merged = added = 0
        for c, j in zip(cand, match):
            c.z -= self.x
            if j < 0:
                self.polys.append(c)
                added += 1
                continue
            m = self.polys[j]                  # keeps its height: the map is the reference
            m.xy = hull_ccw(np.concatenate([m.xy, c.xy]))
            m.area = area(m.xy)
            m.observations += 1
            merged += 1
        return dict(matched=len(offsets), merged=merged, added=added, skipped=skipped,
                    measurement=zk, gain=K, drift_prior=x_prior, drift=self.x, variance=self.P)
