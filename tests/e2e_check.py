"""End-to-end comparison of a frame's planes with the oracle's.

Diffusion agrees to about 1e-7 m, so the FP32 points of the two sides can
differ in the last bit; a single inlier decision near the threshold then
changes the candidate count, after which the two runs draw different
hypotheses and may pick different (equally valid) winners for soft planes
(narrow treads whose refit depends on the slab).  Strict plane parity is
checked at the RANSAC stage, on identical points.  End to end, this checks:
the dominant first plane within the plane tolerance, every oracle plane with
at least `min_big` inliers matched by a GPU plane on the same ground-truth
surface, and the per-pixel labels agreeing on at least 95% of the pixels.
"""
import numpy as np

PLANE_DEG, PLANE_OFF = 0.1, 1e-3


def ang(a, b):
    return np.degrees(np.arccos(np.clip(abs(float(a @ b)), 0.0, 1.0)))


def surface_of(labels, k, plane_id):
    sel = labels == k
    g = plane_id[sel]
    g = g[g >= 0]
    return int(np.bincount(g).argmax()) if g.size else -1


def check_end_to_end(fr, gpu_planes, gpu_labels, orc, min_big=1000):
    """gpu_planes: Planes; gpu_labels: int16 [h, w] numpy; orc: RansacResult."""
    assert len(gpu_planes.planes) >= 1 and len(orc.planes) >= 1
    g0, o0 = gpu_planes.planes[0], orc.planes[0]
    assert ang(g0[:3], o0[:3]) <= PLANE_DEG and abs(g0[3] - o0[3]) <= PLANE_OFF, (g0, o0)
    gpu_surf = {surface_of(gpu_labels, k, fr.plane_id) for k in range(len(gpu_planes.planes))}
    for k in range(len(orc.planes)):
        if orc.n_inliers[k] >= min_big:
            s = surface_of(orc.labels, k, fr.plane_id)
            assert s in gpu_surf, ('oracle plane %d on surface %d not found' % (k, s))
    agree = float((gpu_labels == orc.labels).mean())
    assert agree >= 0.95, agree
    return agree
