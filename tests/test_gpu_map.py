"""End to end on a walk up a staircase: every frame through the GPU path
(diffusion, normals, Canny edges, regions, per-region RANSAC), the regions'
outlines into the map manager with a drifting odometry pose (Sec. III-E)."""
import numpy as np
import pytest
import torch

import synth
from paper_2411_01919_b300 import Params, Pipeline
from paper_2411_01919_b300.mapping import MapManager, region_polygons

pytestmark = pytest.mark.gpu


def test_walk_builds_a_map_of_the_treads_and_tracks_the_drift():
    w, h = 320, 240
    fx, fy, cx, cy = 385.0 * w / 640, 385.0 * w / 640, w / 2, h / 2
    walk = synth.tread_walk(16, 3, n_steps=6, first_y=0.8, drift_sigma=0.0, drift_bias=0.002,
                            vertex_noise=0.0)
    sc = synth.straight_staircase(6, 0.15, 0.28, 1.0, first_riser_y=0.8)
    rng = np.random.Generator(np.random.PCG64(7))
    mm = MapManager()
    p = Params(iters=20, hypotheses=256, thr=0.01, max_planes=4, seed=1)
    with Pipeline(p, w, h, 1) as pipe:
        for k, f in enumerate(walk):
            cam = synth.Camera(w, h, fx, fy, cx, cy, f.pose_true[:3, 3], f.pose_true[:3, :3])
            fr = synth.sense(sc, cam, rng, 0.002, 0.02, True, 'u16')
            z = pipe.diffuse(torch.from_numpy(fr.encoded).cuda())
            P, N, V = pipe.normals(z, cam.intrinsics)
            lab, R = pipe.segment(pipe.canny(N, V), V, 150)
            if R == 0:
                st = mm.integrate(f.pose_odom, [])
                continue
            res = pipe.ransac_regions(P, V, lab, R, 256, k)
            polys = region_polygons(P.cpu().numpy(), lab.cpu().numpy(), res.planes, res.accepted)
            st = mm.integrate(f.pose_odom, polys)
    true_drift = walk[-1].drift
    x, _ = mm.drift()
    assert abs(x - true_drift) < 0.015, (x, true_drift)
    heights = [p[1] for p in mm.polygons() if p[2] > 0.05]
    gt = np.array([0.15 * i for i in range(7)])
    # every sizeable map polygon lies at a true tread (or floor) height, and
    # the near treads are all in the map
    for hh in heights:
        assert np.abs(gt - hh).min() < 0.02, (hh, heights)
    hit = {int(np.argmin(np.abs(gt - hh))) for hh in heights}
    assert {0, 1, 2, 3} <= hit, heights
