"""Seeded synthetic depth frames of staircases (straight and spiral).

This module is the input generator shared by the FP64 oracle and the CUDA path.
It ray-casts analytic scenes (axis-aligned boxes, annular-sector prisms,
cylinders and the floor) through a pinhole camera and returns a depth image
(camera-frame Z, metres), the ground-truth plane of every pixel, sensor noise
and holes, and the encodings a depth sensor delivers (u16 millimetres, FP16
metres, FP32 metres).  It contains none of the method's arithmetic: no
diffusion, no normal estimation, no plane fitting.

The scenes stand in for the paper's RealSense L515 recordings of a stair model
(Sec. III-B, Sec. IV-A), which are not available.  Conventions:

* World frame: x right, y forward, z up; the floor is z = 0.
* Camera frame (OpenCV): x right, y down, z along the optical axis.  A pixel
  (u, v) (u = column, v = row, centres at integer coordinates) looks along
  ((u - cx)/fx, (v - cy)/fy, 1); the depth is the Z coordinate of the hit.
* Planes are stored as (n, d) with n . X + d = 0, |n| = 1, oriented towards the
  camera (d > 0 in the camera frame).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

MAX_RANGE_M = 9.0          # L515-like maximum range; farther hits become holes
U16_MAX = 65535


@dataclass
class Camera:
    w: int
    h: int
    fx: float
    fy: float
    cx: float
    cy: float
    pos: np.ndarray            # (3,) world position
    R: np.ndarray              # (3, 3) camera -> world rotation, columns = cam x, y, z

    @property
    def intrinsics(self):
        return (self.fx, self.fy, self.cx, self.cy)


@dataclass
class Frame:
    """One synthetic depth frame and its ground truth."""
    cam: Camera
    depth_clean: np.ndarray    # (h, w) float64, metres, 0 where the ray hits nothing
    depth: np.ndarray          # (h, w) float64, noisy, 0 = hole
    plane_id: np.ndarray       # (h, w) int32, index into planes, -1 = curved / miss / hole
    planes: np.ndarray         # (P, 4) float64 camera-frame planes (nx, ny, nz, d)
    dtype: str                 # 'u16' | 'f16' | 'f32': the encoding of `encoded`
    encoded: np.ndarray        # (h, w) uint16 mm | float16 m | float32 m
    depth_scale: float = 0.001  # metres per u16 unit
    meta: dict = field(default_factory=dict)

    @property
    def w(self):
        return self.cam.w

    @property
    def h(self):
        return self.cam.h

    def decoded(self) -> np.ndarray:
        """The depth as the sensor delivers it, in metres (float64), 0 = hole."""
        e = self.encoded
        if self.dtype == 'u16':
            return e.astype(np.float64) * self.depth_scale
        return e.astype(np.float64)


# ----------------------------------------------------------------------------
# camera construction
# ----------------------------------------------------------------------------

def look_rotation(yaw: float, pitch_down: float) -> np.ndarray:
    """Camera->world rotation for a camera with heading `yaw` (radians, 0 = +y,
    positive turns towards +x) pitched down by `pitch_down` radians."""
    cy_, sy_ = np.cos(yaw), np.sin(yaw)
    cp, sp = np.cos(pitch_down), np.sin(pitch_down)
    fwd = np.array([sy_ * cp, cy_ * cp, -sp])
    right = np.array([cy_, -sy_, 0.0])
    down = np.cross(fwd, right)
    return np.stack([right, down, fwd], axis=1)


def make_camera(w, h, fx, fy, cx, cy, pos, yaw=0.0, pitch_down=np.pi / 4):
    return Camera(w, h, float(fx), float(fy), float(cx), float(cy),
                  np.asarray(pos, dtype=np.float64), look_rotation(yaw, pitch_down))


def pixel_rays(cam: Camera):
    """World-frame ray directions scaled so that the camera Z of the direction is 1."""
    u = np.arange(cam.w, dtype=np.float64)
    v = np.arange(cam.h, dtype=np.float64)
    uu, vv = np.meshgrid(u, v)
    dc = np.stack([(uu - cam.cx) / cam.fx, (vv - cam.cy) / cam.fy, np.ones_like(uu)], axis=-1)
    return dc @ cam.R.T      # (h, w, 3)


# ----------------------------------------------------------------------------
# scene primitives: every primitive returns (t, face_key) arrays; t = inf on miss
# ----------------------------------------------------------------------------

class Scene:
    """A union of solids.  Each planar face carries a world plane (n_w, d_w)."""

    def __init__(self):
        self.faces = []          # list of (n_w (3,), d_w) or None for curved faces
        self.solids = []         # list of callables (o, d) -> (t, face_index)

    def add_face(self, n_w, d_w):
        self.faces.append((np.asarray(n_w, dtype=np.float64), float(d_w)))
        return len(self.faces) - 1

    def add_curved(self):
        self.faces.append(None)
        return len(self.faces) - 1

    # -- floor ---------------------------------------------------------------
    def add_floor(self):
        fid = self.add_face([0.0, 0.0, 1.0], 0.0)

        def hit(o, d):
            with np.errstate(divide='ignore', invalid='ignore'):
                t = np.where(d[..., 2] < 0, -o[2] / d[..., 2], np.inf)
            return t, np.full(t.shape, fid, dtype=np.int32)
        self.solids.append(hit)

    # -- axis-aligned box ----------------------------------------------------
    def add_box(self, lo, hi):
        lo = np.asarray(lo, dtype=np.float64)
        hi = np.asarray(hi, dtype=np.float64)
        # face ids: axis a, side 0 = min face (outward normal -e_a), 1 = max face
        fids = np.zeros((3, 2), dtype=np.int32)
        for a in range(3):
            e = np.zeros(3)
            e[a] = 1.0
            fids[a, 0] = self.add_face(-e, lo[a])      # -x_a + lo = 0
            fids[a, 1] = self.add_face(e, -hi[a])      #  x_a - hi = 0

        def hit(o, d):
            with np.errstate(divide='ignore', invalid='ignore'):
                inv = 1.0 / d
                t1 = (lo - o) * inv
                t2 = (hi - o) * inv
            tmin = np.minimum(t1, t2)
            tmax = np.maximum(t1, t2)
            tmin = np.nan_to_num(tmin, nan=-np.inf)
            tmax = np.nan_to_num(tmax, nan=np.inf)
            tnear = tmin.max(axis=-1)
            tfar = tmax.min(axis=-1)
            axis = tmin.argmax(axis=-1)
            ok = (tnear <= tfar) & (tnear > 0)
            side = np.take_along_axis(d, axis[..., None], axis=-1)[..., 0] < 0  # entering max face
            fid = fids[axis, side.astype(np.int64)]
            return np.where(ok, tnear, np.inf), fid
        self.solids.append(hit)

    # -- annular sector prism (spiral step) ----------------------------------
    def add_sector_prism(self, axis_xy, r_in, r_out, th_a, th_b, z_top):
        ax, ay = axis_xy
        top = self.add_face([0.0, 0.0, 1.0], -z_top)
        # radial faces: the plane through the axis at angle th; outward normal
        # points away from the sector's interior
        na = np.array([np.sin(th_a), -np.cos(th_a), 0.0])
        nb = np.array([-np.sin(th_b), np.cos(th_b), 0.0])
        A = np.array([ax, ay, 0.0])
        fa = self.add_face(na, -na @ A)
        fb = self.add_face(nb, -nb @ A)
        outer = self.add_curved()
        span = th_b - th_a

        def in_sector(x, y):
            phi = np.arctan2(y - ay, x - ax)
            return np.mod(phi - th_a, 2 * np.pi) <= span

        def hit(o, d):
            best = np.full(d.shape[:-1], np.inf)
            fid = np.full(d.shape[:-1], -1, dtype=np.int32)
            with np.errstate(divide='ignore', invalid='ignore'):
                # top face
                t = (z_top - o[2]) / d[..., 2]
                X = o + t[..., None] * d
                rr = np.hypot(X[..., 0] - ax, X[..., 1] - ay)
                ok = (t > 0) & (d[..., 2] < 0) & (rr >= r_in) & (rr <= r_out) & \
                    in_sector(X[..., 0], X[..., 1])
                upd = ok & (t < best)
                best = np.where(upd, t, best)
                fid = np.where(upd, top, fid)
                # radial faces
                for th, nf, f in ((th_a, na, fa), (th_b, nb, fb)):
                    den = d @ nf
                    t = -((o - A) @ nf) / den
                    X = o + t[..., None] * d
                    rho = (X[..., 0] - ax) * np.cos(th) + (X[..., 1] - ay) * np.sin(th)
                    ok = (t > 0) & (den < 0) & (rho >= r_in) & (rho <= r_out) & \
                        (X[..., 2] >= 0) & (X[..., 2] <= z_top)
                    upd = ok & (t < best)
                    best = np.where(upd, t, best)
                    fid = np.where(upd, f, fid)
                # outer cylinder (entry root)
                ox, oy = o[0] - ax, o[1] - ay
                a = d[..., 0] ** 2 + d[..., 1] ** 2
                b = 2 * (ox * d[..., 0] + oy * d[..., 1])
                c = ox * ox + oy * oy - r_out * r_out
                disc = b * b - 4 * a * c
                t = (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a)
                X = o + t[..., None] * d
                ok = (disc >= 0) & (t > 0) & (X[..., 2] >= 0) & (X[..., 2] <= z_top) & \
                    in_sector(X[..., 0], X[..., 1])
                upd = ok & (t < best)
                best = np.where(upd, t, best)
                fid = np.where(upd, outer, fid)
            return best, fid
        self.solids.append(hit)

    # -- vertical cylinder (spiral column) -----------------------------------
    def add_column(self, axis_xy, r, z_top):
        ax, ay = axis_xy
        side = self.add_curved()
        top = self.add_face([0.0, 0.0, 1.0], -z_top)

        def hit(o, d):
            best = np.full(d.shape[:-1], np.inf)
            fid = np.full(d.shape[:-1], -1, dtype=np.int32)
            with np.errstate(divide='ignore', invalid='ignore'):
                ox, oy = o[0] - ax, o[1] - ay
                a = d[..., 0] ** 2 + d[..., 1] ** 2
                b = 2 * (ox * d[..., 0] + oy * d[..., 1])
                c = ox * ox + oy * oy - r * r
                disc = b * b - 4 * a * c
                t = (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a)
                z = o[2] + t * d[..., 2]
                ok = (disc >= 0) & (t > 0) & (z >= 0) & (z <= z_top)
                best = np.where(ok, t, best)
                fid = np.where(ok, side, fid)
                t = (z_top - o[2]) / d[..., 2]
                X = o + t[..., None] * d
                ok = (t > 0) & (d[..., 2] < 0) & (np.hypot(X[..., 0] - ax, X[..., 1] - ay) <= r) & (t < best)
                best = np.where(ok, t, best)
                fid = np.where(ok, top, fid)
            return best, fid
        self.solids.append(hit)

    # -- rendering -----------------------------------------------------------
    def render(self, cam: Camera):
        d = pixel_rays(cam)
        o = cam.pos
        best = np.full(d.shape[:-1], np.inf)
        fid = np.full(d.shape[:-1], -1, dtype=np.int32)
        for solid in self.solids:
            t, f = solid(o, d)
            upd = t < best
            best = np.where(upd, t, best)
            fid = np.where(upd, f, fid)
        miss = ~np.isfinite(best) | (best > MAX_RANGE_M)
        depth = np.where(miss, 0.0, best)
        fid = np.where(miss, -1, fid)
        return depth, fid

    def camera_planes(self, cam: Camera):
        """All planar faces expressed in the camera frame, oriented to the camera.
        Coplanar faces (same plane within 1e-9) share one entry."""
        out, remap = [], {}
        for i, f in enumerate(self.faces):
            if f is None:
                continue
            n_w, d_w = f
            n_c = cam.R.T @ n_w
            d_c = n_w @ cam.pos + d_w
            if d_c < 0:
                n_c, d_c = -n_c, -d_c
            key = None
            for j, p in enumerate(out):
                if np.allclose(p[:3], n_c, atol=1e-9) and abs(p[3] - d_c) < 1e-9:
                    key = j
                    break
            if key is None:
                out.append(np.r_[n_c, d_c])
                key = len(out) - 1
            remap[i] = key
        return np.array(out).reshape(-1, 4), remap


# ----------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------

def straight_staircase(n_steps, rise, tread, width, first_riser_y, landing_depth=1.0,
                       wall_height=3.0) -> Scene:
    """Floor, `n_steps` risers starting `first_riser_y` ahead of the origin, a
    landing `landing_depth` deep on top of the last step and a back wall at the
    landing's far edge."""
    s = Scene()
    s.add_floor()
    y_end = first_riser_y + (n_steps - 1) * tread + landing_depth
    for k in range(1, n_steps + 1):
        y0 = first_riser_y + (k - 1) * tread
        s.add_box([-width / 2, y0, 0.0], [width / 2, y_end, k * rise])
    s.add_box([-3.0, y_end, 0.0], [3.0, y_end + 0.2, wall_height])
    return s


def spiral_staircase(n_steps, step_deg, rise, r_in, r_out, axis_xy=(0.0, 0.0),
                     theta0=0.0, column_height=3.5) -> Scene:
    """Floor, a central column of radius `r_in` and `n_steps` annular-sector
    steps (solid from the floor to their tread) ascending counter-clockwise."""
    s = Scene()
    s.add_floor()
    dth = np.deg2rad(step_deg)
    for k in range(n_steps):
        s.add_sector_prism(axis_xy, r_in, r_out, theta0 + k * dth, theta0 + (k + 1) * dth,
                           (k + 1) * rise)
    s.add_column(axis_xy, r_in, column_height)
    return s


# ----------------------------------------------------------------------------
# sensor model
# ----------------------------------------------------------------------------

def _edge_bands(depth_clean, jump=0.05, radius=2):
    """Pixels within Chebyshev distance `radius` of a 4-neighbour depth jump."""
    h, w = depth_clean.shape
    J = np.zeros((h, w), dtype=bool)
    dx = np.abs(np.diff(depth_clean, axis=1)) > jump
    dy = np.abs(np.diff(depth_clean, axis=0)) > jump
    J[:, :-1] |= dx
    J[:, 1:] |= dx
    J[:-1, :] |= dy
    J[1:, :] |= dy
    out = np.zeros_like(J)
    P = np.pad(J, radius)
    for oy in range(2 * radius + 1):
        for ox in range(2 * radius + 1):
            out |= P[oy:oy + h, ox:ox + w]
    return out


def render_gt(scene: Scene, cam: Camera):
    """Noise-free depth, per-pixel GT plane index and the camera-frame planes."""
    depth_clean, fid = scene.render(cam)
    planes, remap = scene.camera_planes(cam)
    pid = np.full(fid.shape, -1, dtype=np.int32)
    for i, j in remap.items():
        pid[fid == i] = j
    return depth_clean, pid, planes


def sense(scene: Scene, cam: Camera, rng: np.random.Generator, sigma_coeff: float,
          hole_frac: float, edge_bands: bool, dtype: str, depth_scale=0.001,
          meta=None, rendered=None) -> Frame:
    depth_clean, pid, planes = rendered if rendered is not None else render_gt(scene, cam)
    pid = pid.copy()
    valid = depth_clean > 0
    z = depth_clean + rng.standard_normal(depth_clean.shape) * (sigma_coeff * depth_clean ** 2)
    z = np.where(valid, np.maximum(z, 1e-3), 0.0)
    holes = rng.random(depth_clean.shape) < hole_frac
    if edge_bands:
        holes |= _edge_bands(depth_clean)
    z = np.where(holes, 0.0, z)
    if dtype == 'u16':
        enc = np.clip(np.rint(z / depth_scale), 0, U16_MAX).astype(np.uint16)
    elif dtype == 'f16':
        enc = z.astype(np.float16)
    elif dtype == 'f32':
        enc = z.astype(np.float32)
    else:
        raise ValueError(dtype)
    pid = np.where(holes | ~valid, -1, pid)
    return Frame(cam, depth_clean, z, pid, planes, dtype, enc, depth_scale, meta or {})


# ----------------------------------------------------------------------------
# the workloads (sizes and parameters of the five benchmark configurations)
# ----------------------------------------------------------------------------

def frame_c1(seed: int) -> Frame:
    """160x120 FP32 straight staircase: 3 steps (rise 0.15, tread 0.28, width 1.0),
    camera 1.0 m above the floor pitched 45 deg down, sigma = 0.0015 z^2, 1% holes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cam = make_camera(160, 120, 120.0, 120.0, 80.0, 60.0, [0.0, 0.0, 1.0], 0.0, np.pi / 4)
    sc = straight_staircase(3, 0.15, 0.28, 1.0, first_riser_y=0.6)
    return sense(sc, cam, rng, 0.0015, 0.01, False, 'f32', meta={'config': 'c1', 'seed': seed})


_C2_CACHE = {}


def frame_c2(seed: int) -> Frame:
    """640x480 u16-mm straight staircase: 6 steps + floor + landing,
    sigma = 0.002 z^2, 2% random holes plus 5-pixel bands at depth edges.
    The geometry does not depend on the seed; noise and holes do."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cam = make_camera(640, 480, 385.0, 385.0, 320.0, 240.0, [0.0, 0.0, 1.0], 0.0, np.pi / 4)
    sc = straight_staircase(6, 0.15, 0.28, 1.0, first_riser_y=0.8)
    if 'gt' not in _C2_CACHE:
        _C2_CACHE['gt'] = render_gt(sc, cam)
    return sense(sc, cam, rng, 0.002, 0.02, True, 'u16', meta={'config': 'c2', 'seed': seed},
                 rendered=_C2_CACHE['gt'])


def frame_straight(seed: int, w: int, h: int, sigma_coeff: float = 0.002,
                   hole_frac: float = 0.02, dtype: str = 'u16') -> Frame:
    """The 640x480 straight staircase scene (6 steps + floor + landing, camera
    1.0 m high pitched 45 deg down) seen at w x h (intrinsics scaled with the
    width) with noise sigma = sigma_coeff z^2, random holes and 5-pixel hole
    bands at depth edges.  Used for resolution and noise sweeps."""
    rng = np.random.Generator(np.random.PCG64([seed, w, h]))
    fx, fy, cx, cy = _scaled_intrinsics(w, h)
    cam = make_camera(w, h, fx, fy, cx, cy, [0.0, 0.0, 1.0], 0.0, np.pi / 4)
    sc = straight_staircase(6, 0.15, 0.28, 1.0, first_riser_y=0.8)
    return sense(sc, cam, rng, sigma_coeff, hole_frac, True, dtype,
                 meta={'config': 'straight', 'seed': seed, 'sigma_coeff': sigma_coeff})


def _spiral_camera(rng, w, h, fx, fy, cx, cy, height=1.2):
    dist = rng.uniform(2.2, 2.8)
    phi = rng.uniform(-0.3, 0.3) - np.pi / 2          # camera stands on the -y side
    pos = np.array([dist * np.cos(phi), dist * np.sin(phi), height])
    yaw = np.arctan2(-pos[0], -pos[1]) + rng.uniform(-0.1, 0.1)
    pitch = np.deg2rad(rng.uniform(30.0, 40.0))
    return make_camera(w, h, fx, fy, cx, cy, pos, yaw, pitch)


def frame_c3(seed: int) -> Frame:
    """848x480 FP16 spiral staircase: 12 steps of 20 deg, rise 0.17, radii 0.3-1.1,
    seeded camera pose at 1.2 m height; sigma = 0.002 z^2, 2% holes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cam = _spiral_camera(rng, 848, 480, 425.0, 425.0, 424.0, 240.0)
    sc = spiral_staircase(12, 20.0, 0.17, 0.3, 1.1, theta0=-np.pi / 2 - 0.35)
    return sense(sc, cam, rng, 0.002, 0.02, False, 'f16', meta={'config': 'c3', 'seed': seed})


RES_C4 = [(320, 240), (640, 480), (848, 480), (1280, 720)]
RES_C5 = [(424, 240), (640, 480), (848, 480), (1280, 720)]


def _scaled_intrinsics(w, h):
    f = 385.0 * w / 640.0
    return f, f, w / 2.0, h / 2.0


def _random_scene(rng):
    rise = rng.uniform(0.12, 0.20)
    tread = rng.uniform(0.22, 0.32)
    if rng.random() < 0.5:
        return 'straight', straight_staircase(int(rng.integers(3, 8)), rise, tread,
                                              rng.uniform(0.9, 1.4), rng.uniform(0.6, 1.0))
    step_deg = np.rad2deg(tread / 0.7)
    return 'spiral', spiral_staircase(int(rng.integers(8, 13)), step_deg, rise, 0.3, 1.1,
                                      theta0=-np.pi / 2 - 0.35)


def frame_c4(seed: int, index: int) -> Frame:
    """One frame of the 64-frame batched workload: resolution drawn from RES_C4,
    straight or spiral staircase with seeded geometry, FP16 storage,
    sigma = 0.002 z^2, 2% holes.  `meta['iters']` is the frame's diffusion
    iteration count, drawn from [20, 40]."""
    rng = np.random.Generator(np.random.PCG64([seed, index]))
    w, h = RES_C4[int(rng.integers(len(RES_C4)))]
    kind, sc = _random_scene(rng)
    fx, fy, cx, cy = _scaled_intrinsics(w, h)
    if kind == 'straight':
        cam = make_camera(w, h, fx, fy, cx, cy, [0.0, 0.0, rng.uniform(0.9, 1.1)], 0.0,
                          np.deg2rad(rng.uniform(40, 50)))
    else:
        cam = _spiral_camera(rng, w, h, fx, fy, cx, cy)
    iters = int(rng.integers(20, 41))
    return sense(sc, cam, rng, 0.002, 0.02, False, 'f16',
                 meta={'config': 'c4', 'seed': seed, 'index': index, 'iters': iters, 'scene': kind})


def frame_c5(stream: int, k: int, seed: int = 0) -> Frame:
    """Frame k of simulated camera stream `stream`: the stream's resolution is
    fixed (drawn from RES_C5), its scene is a seeded staircase and the camera
    advances 5 cm per frame (wrapping every 20 frames so the stairs stay in view)."""
    srng = np.random.Generator(np.random.PCG64([seed, 1000 + stream]))
    w, h = RES_C5[int(srng.integers(len(RES_C5)))]
    kind, sc = _random_scene(srng)
    fx, fy, cx, cy = _scaled_intrinsics(w, h)
    step = 0.05 * (k % 20)
    if kind == 'straight':
        cam = make_camera(w, h, fx, fy, cx, cy, [0.0, -0.5 + step, 1.0], 0.0, np.pi / 4)
    else:
        base = _spiral_camera(srng, w, h, fx, fy, cx, cy)
        fwd = base.R[:, 2].copy()
        fwd[2] = 0.0
        fwd /= np.linalg.norm(fwd)
        cam = Camera(w, h, fx, fy, cx, cy, base.pos + (step - 0.5) * fwd, base.R)
    frng = np.random.Generator(np.random.PCG64([seed, 1000 + stream, k]))
    return sense(sc, cam, frng, 0.002, 0.02, False, 'f16',
                 meta={'config': 'c5', 'stream': stream, 'k': k, 'iters': 30, 'scene': kind})


def plane_frame(w, h, fx, fy, cx, cy, n, d, dtype='f32') -> Frame:
    """Noise-free depth of the single camera-frame plane n . X + d = 0 (rays that
    hit it behind the camera or beyond range become holes).  Used to pin normals."""
    n = np.asarray(n, dtype=np.float64)
    n = n / np.linalg.norm(n)
    u = np.arange(w, dtype=np.float64)
    v = np.arange(h, dtype=np.float64)
    uu, vv = np.meshgrid(u, v)
    den = n[0] * (uu - cx) / fx + n[1] * (vv - cy) / fy + n[2]
    with np.errstate(divide='ignore', invalid='ignore'):
        z = -d / den
    z = np.where((z > 0) & (z <= MAX_RANGE_M) & np.isfinite(z), z, 0.0)
    cam = Camera(w, h, fx, fy, cx, cy, np.zeros(3), np.eye(3))
    pid = np.where(z > 0, 0, -1).astype(np.int32)
    nn = n if d > 0 else -n
    planes = np.array([[*nn, abs(d)]])
    enc = z.astype({'f32': np.float32, 'f16': np.float16}[dtype]) if dtype != 'u16' else \
        np.clip(np.rint(z * 1000), 0, U16_MAX).astype(np.uint16)
    return Frame(cam, z, z.copy(), pid, planes, dtype, enc)


def _c5_job(args):
    stream, k, seed = args
    f = frame_c5(stream, k, seed)
    return stream, k, f


def stream_pool(n_streams: int, poses: int, seed: int = 0, workers: int = 0):
    """Frames of `n_streams` simulated cameras at `poses` successive poses (5 cm
    apart), rendered in a pool of spawned worker processes (safe to call after
    CUDA is initialised).  Returns {stream: [Frame, ...]}."""
    import multiprocessing as mp
    jobs = [(s, k, seed) for s in range(n_streams) for k in range(poses)]
    out = {s: [None] * poses for s in range(n_streams)}
    if workers and workers > 1:
        ctx = mp.get_context('spawn')
        with ctx.Pool(workers) as pool:
            for s, k, f in pool.imap_unordered(_c5_job, jobs):
                out[s][k] = f
    else:
        for job in jobs:
            s, k, f = _c5_job(job)
            out[s][k] = f
    return out


def _render_job(job):
    name, args = job
    return globals()[name](*args)


def render_many(name: str, arg_list, workers: int = 0):
    """[name(*args) for args in arg_list] for one of this module's frame
    functions (e.g. 'frame_c3'), rendered in a pool of spawned worker
    processes when workers > 1 (safe to call after CUDA is initialised)."""
    import multiprocessing as mp
    jobs = [(name, tuple(a)) for a in arg_list]
    if workers and workers > 1 and len(jobs) > 1:
        with mp.get_context('spawn').Pool(min(workers, len(jobs))) as pool:
            return pool.map(_render_job, jobs, chunksize=1)
    return [_render_job(j) for j in jobs]
