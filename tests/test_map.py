"""The polygon map manager (Sec. III-E, Eq. 4-10): its oracle pinned to closed
forms, and the native implementation in libpm (host code) against the oracle.

Pins: the Kalman variance and gain follow the scalar Riccati recursion to its
closed-form steady state; the first drift update and compensation in closed
form; a large sigma_p / sigma_m ratio lets the measurement dominate (as the
section advises); the 5 cm tolerance boundary (Eq. 5); overlap areas of
rectangles in closed form and of random convex polygons by Monte Carlo;
non-horizontal polygons skipped; drift recovery after a step."""
import math

import numpy as np
import pytest

import synth
from oracle import mapping as om
from paper_2411_01919_b300 import PmError
from paper_2411_01919_b300.mapping import MapManager, MapParams, region_polygons

SP, SM, P0 = 1e-5, 1e-4, 1e-4


def square_polygon(z, cx=0.0, cy=2.0, half=0.3, tilt_deg=0.0):
    """A horizontal (or tilted about x) square seen by a camera at the origin
    looking down the map's -z (camera = map frame): (n, d, vertices)."""
    t = math.radians(tilt_deg)
    n = np.array([0.0, -math.sin(t), math.cos(t)])
    V = []
    for sx, sy in ((-1, -1), (1, -1), (1, 1), (-1, 1)):
        x, y = cx + sx * half, cy + sy * half
        V.append([x, y, z + math.tan(t) * (y - cy)])
    V = np.array(V)
    return n, float(-n @ V.mean(axis=0)), V


def shifted(z):
    T = np.eye(4)
    T[2, 3] = z
    return T


def test_kalman_variance_reaches_the_riccati_steady_state():
    o = om.MapOracle(sigma_p=SP, sigma_m=SM, P=P0)
    o.integrate(np.eye(4), [square_polygon(0.0)])
    Ks = []
    for k in range(200):
        st = o.integrate(shifted(0.001 * (k % 3)), [square_polygon(0.0)])
        assert st['matched'] == 1
        Ks.append(st['gain'])
    p_inf = (-SP + math.sqrt(SP * SP + 4 * SP * SM)) / 2
    k_inf = (p_inf + SP) / (p_inf + SP + SM)
    assert o.P == pytest.approx(p_inf, rel=1e-9)
    assert Ks[-1] == pytest.approx(k_inf, rel=1e-9)
    assert all(a >= b for a, b in zip(Ks, Ks[1:]))     # from P0 above the steady state


def test_first_update_and_compensation_in_closed_form():
    c = 0.02
    o = om.MapOracle(sigma_p=SP, sigma_m=SM, P=P0)
    o.integrate(np.eye(4), [square_polygon(0.0)])
    st = o.integrate(shifted(c), [square_polygon(0.0, cy=2.4)])
    P1 = P0 + 2 * SP                  # one prediction per frame: frames 0 and 1
    K = P1 / (P1 + SM)
    assert st['measurement'] == pytest.approx(c, abs=1e-15)
    assert st['gain'] == pytest.approx(K, rel=1e-12)
    assert st['drift'] == pytest.approx(K * c, rel=1e-12)
    assert st['variance'] == pytest.approx((1 - K) * P1, rel=1e-12)
    assert o.polys[0].z == 0.0                            # the map keeps its height
    assert o.polys[0].area == pytest.approx(0.6 * 1.0, rel=1e-12)   # footprint grew to the hull


def test_measurement_dominates_when_process_noise_is_large():
    o = om.MapOracle(sigma_p=1.0, sigma_m=1e-6, P=0.0)
    o.integrate(np.eye(4), [square_polygon(0.0)])
    st = o.integrate(shifted(0.03), [square_polygon(0.0)])
    assert st['gain'] > 0.999998 and st['drift'] == pytest.approx(0.03, rel=1e-5)


@pytest.mark.parametrize('dz,merges', [(0.0499, True), (0.04999, True), (0.05001, False),
                                       (0.0501, False), (-0.04999, True), (-0.05001, False)])
def test_tolerance_boundary(dz, merges):
    for impl in ('oracle', 'native'):
        m = om.MapOracle() if impl == 'oracle' else MapManager()
        m.integrate(np.eye(4), [square_polygon(1.0)])
        st = m.integrate(np.eye(4), [square_polygon(1.0 + dz)])
        assert (st['matched'] == 1) == merges, impl
        n = len(m.polys) if impl == 'oracle' else len(m)
        assert n == (1 if merges else 2)


def test_matching_uses_the_drift_estimate():
    """Eq. 4-5 compare heights after removing the drift estimated so far: with
    the estimate near 4 cm, a polygon 8.5 cm above its map match still merges."""
    for impl in ('oracle', 'native'):
        m = om.MapOracle() if impl == 'oracle' else MapManager()
        m.integrate(np.eye(4), [square_polygon(0.0)])
        for _ in range(60):
            m.integrate(shifted(0.04), [square_polygon(0.0)])
        st = m.integrate(shifted(0.085), [square_polygon(0.0)])
        assert st['drift_prior'] == pytest.approx(0.04, abs=1e-6), impl
        assert st['matched'] == 1 and st['measurement'] == pytest.approx(0.085), impl


def test_overlap_is_required_for_a_merge():
    for m in (om.MapOracle(), MapManager()):
        m.integrate(np.eye(4), [square_polygon(0.5, cx=0.0)])
        st = m.integrate(np.eye(4), [square_polygon(0.5, cx=0.61)])    # 1 cm gap
        assert st['matched'] == 0 and st['added'] == 1


def test_rectangle_overlap_in_closed_form():
    rng = np.random.default_rng(0)
    for _ in range(200):
        x0, y0 = rng.uniform(-1, 1, 2)
        w0, h0 = rng.uniform(0.1, 1, 2)
        x1, y1 = rng.uniform(-1, 1, 2)
        w1, h1 = rng.uniform(0.1, 1, 2)
        rect = lambda x, y, w, h: np.array([[x, y], [x + w, y], [x + w, y + h], [x, y + h]])
        want = max(0, min(x0 + w0, x1 + w1) - max(x0, x1)) * max(0, min(y0 + h0, y1 + h1) - max(y0, y1))
        got = om.clip_area(rect(x0, y0, w0, h0), rect(x1, y1, w1, h1))
        assert got == pytest.approx(want, abs=1e-12)


def test_convex_overlap_by_monte_carlo():
    rng = np.random.default_rng(1)
    for _ in range(5):
        a = om.hull_ccw(rng.normal(0, 1, (12, 2)))
        b = om.hull_ccw(rng.normal(0.5, 1, (12, 2)))
        got = om.clip_area(a, b)
        q = rng.uniform(-4, 4, (400000, 2))

        def inside(poly, q):
            ok = np.ones(len(q), bool)
            for e in range(len(poly)):
                p0, p1 = poly[e], poly[(e + 1) % len(poly)]
                ok &= (p1[0] - p0[0]) * (q[:, 1] - p0[1]) - (p1[1] - p0[1]) * (q[:, 0] - p0[0]) >= 0
            return ok
        mc = (inside(a, q) & inside(b, q)).mean() * 64.0
        assert got == pytest.approx(mc, abs=0.05)


def test_non_horizontal_polygons_are_skipped():
    for m in (om.MapOracle(), MapManager()):
        st = m.integrate(np.eye(4), [square_polygon(0.2, tilt_deg=30.0), square_polygon(0.0)])
        assert st['skipped'] == 1 and st['added'] == 1


def test_drift_recovered_after_a_step_and_old_heights_kept():
    walk = synth.tread_walk(30, 1, drift_sigma=0.0, vertex_noise=0.0)
    o = om.MapOracle()
    for k, f in enumerate(walk):
        T = f.pose_true.copy()
        if k >= 10:
            T[2, 3] += 0.03
        st = o.integrate(T, f.polygons)
    assert abs(st['drift'] - 0.03) < 0.005
    # treads already in the map before the step keep their true heights
    first = synth.tread_walk(10, 1, drift_sigma=0.0, vertex_noise=0.0)
    seen = sorted({i for f in first for i in f.tread_ids})
    for i in seen:
        want = 0.0 if i < 0 else 0.15 * (i + 1)
        assert min(abs(p.z - want) for p in o.polys) < 1e-9


def compare(a, b):
    for k in ('matched', 'merged', 'added', 'skipped'):
        assert a[k] == b[k], k
    for k in ('measurement', 'gain', 'drift_prior', 'drift', 'variance'):
        assert b[k] == pytest.approx(a[k], rel=1e-9, abs=1e-15), k


@pytest.mark.parametrize('seed,sigma,bias', [(0, 0.003, 0.0), (1, 0.002, 0.001), (2, 0.0, 0.002)])
def test_native_map_manager_equals_oracle(seed, sigma, bias):
    walk = synth.tread_walk(50, seed, drift_sigma=sigma, drift_bias=bias)
    o, m = om.MapOracle(), MapManager()
    rng = np.random.default_rng(seed)
    for f in walk:
        polys = list(f.polygons)
        if rng.random() < 0.3:                     # a riser: skipped by both
            polys.append(square_polygon(0.3, tilt_deg=85.0))
        compare(o.integrate(f.pose_odom, polys), m.integrate(f.pose_odom, polys))
    assert len(m) == len(o.polys)
    for i, p in enumerate(o.polys):
        xy, z, a, obs = m.polygon(i)
        assert z == pytest.approx(p.z, abs=1e-12)
        assert a == pytest.approx(p.area, rel=1e-9)
        assert obs == p.observations
        assert np.allclose(np.sort(xy, axis=0), np.sort(p.xy, axis=0), atol=1e-9)
    x, P = m.drift()
    assert x == pytest.approx(o.x, rel=1e-9) and P == pytest.approx(o.P, rel=1e-9)


def test_region_polygons_outline_planar_regions():
    """A region of points on a plane becomes its convex outline on the plane."""
    h, w = 40, 60
    vv, uu = np.mgrid[0:h, 0:w]
    P = np.stack([(uu - 30) * 0.01, (vv - 20) * 0.01, np.full((h, w), 1.5)]).astype(np.float32)
    labels = np.full((h, w), -1, np.int32)
    labels[5:30, 10:50] = 0
    planes = np.array([[0.0, 0.0, 2.0, -3.0]])
    polys = region_polygons(P, labels, planes, np.array([True]))
    assert len(polys) == 1
    n, d, V = polys[0]
    assert np.allclose(n, [0, 0, 1]) and d == pytest.approx(-1.5)
    assert len(V) == 4 and np.allclose(V[:, 2], 1.5)
    xs, ys = np.sort(np.unique(V[:, 0].round(6))), np.sort(np.unique(V[:, 1].round(6)))
    assert np.allclose(xs, [-0.2, 0.19]) and np.allclose(ys, [-0.15, 0.09])


def test_argument_errors():
    with pytest.raises(PmError):
        MapManager(MapParams(drift_tolerance_m=0.0))
    with pytest.raises(PmError):
        MapManager(MapParams(sigma_m=0.0))
    m = MapManager()
    with pytest.raises(PmError):
        m.integrate(np.eye(4), [(np.array([0, 0, 1.0]), 0.0, np.zeros((2, 3)))])
    with pytest.raises(PmError):
        m.polygon(0)
    assert m.integrate(np.eye(4), [])['added'] == 0
