"""Seeded camera walks over a staircase for the map manager: the true camera
pose, the odometry pose with a vertical random-walk drift, and the stair
treads the camera sees, as polygons in the camera frame (input generator:
no part of the method's arithmetic)."""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Tuple

import numpy as np


@dataclass
class WalkFrame:
    pose_true: np.ndarray          # 4x4 map <- camera
    pose_odom: np.ndarray          # the same with the odometry's vertical drift
    drift: float                   # pose_odom z - pose_true z
    polygons: List[Tuple[np.ndarray, float, np.ndarray]]   # (n, d, vertices [k, 3]) camera frame
    tread_ids: List[int]


def _camera_rotation(pitch_down: float) -> np.ndarray:
    """Camera looking along +y of the map, pitched down; camera axes x right,
    y down, z forward."""
    c, s = np.cos(pitch_down), np.sin(pitch_down)
    fwd = np.array([0.0, c, -s])
    right = np.array([1.0, 0.0, 0.0])
    down = np.cross(fwd, right)
    return np.stack([right, down, fwd], axis=1)          # columns: camera axes in the map


def tread_walk(n_frames: int, seed: int, n_steps: int = 8, rise: float = 0.15,
               tread: float = 0.28, width: float = 1.0, first_y: float = 1.0,
               step_y: float = 0.05, drift_sigma: float = 0.003, drift_bias: float = 0.0,
               vertex_noise: float = 0.002, view: Tuple[float, float] = (0.4, 2.2),
               pitch_down: float = np.pi / 4, height: float = 1.0) -> List[WalkFrame]:
    """A camera `height` above the floor walks up the y axis by `step_y` per
    frame (rising with the stairs it has passed).  Tread i is the rectangle
    x in [-w/2, w/2], y in [first_y + i tread, first_y + (i+1) tread] at height
    (i+1) rise; the floor (y < first_y) is tread -1 at height 0.  Each frame
    sees the part of every tread inside y in [y_cam + view[0], y_cam + view[1]]
    (kept if at least 5 cm long), corners jittered by `vertex_noise`.  The
    odometry drifts vertically by a random walk (per-frame sigma
    `drift_sigma`, mean `drift_bias`)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    R = _camera_rotation(pitch_down)
    treads = [(-1, -5.0, first_y, 0.0)] + [
        (i, first_y + i * tread, first_y + (i + 1) * tread, (i + 1) * rise) for i in range(n_steps)]
    out, drift = [], 0.0
    for k in range(n_frames):
        yc = k * step_y
        passed = max(0, min(n_steps, int(np.floor((yc - first_y) / tread)) + 1)) if yc >= first_y else 0
        t = np.array([0.0, yc, height + passed * rise])
        T = np.eye(4)
        T[:3, :3] = R
        T[:3, 3] = t
        if k > 0:
            drift += drift_bias + drift_sigma * rng.standard_normal()
        To = T.copy()
        To[2, 3] += drift
        polys, ids = [], []
        for tid, y0, y1, z in treads:
            a, b = max(y0, yc + view[0]), min(y1, yc + view[1])
            if b - a < 0.05:
                continue
            corners = np.array([[-width / 2, a, z], [width / 2, a, z], [width / 2, b, z],
                                [-width / 2, b, z]])
            corners[:, :2] += vertex_noise * rng.standard_normal((4, 2))
            Vc = (R.T @ (corners - t).T).T                   # map -> camera
            n_c = R.T @ np.array([0.0, 0.0, 1.0])
            d_c = -float(n_c @ Vc[0])
            polys.append((n_c, d_c, Vc))
            ids.append(tid)
        out.append(WalkFrame(T, To, drift, polys, ids))
    return out
