"""Host-side checks of the C ABI (no GPU): the library loads, exports every
function include/pm.h declares, struct layouts match, and argument errors are
reported before anything touches the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2411_01919_b300 as pm
from paper_2411_01919_b300 import _ffi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, 'include', 'pm.h')


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r'/\*.*?\*/', '', src, flags=re.S)
    names = re.findall(r'^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?[\s\*]+(pm_[a-z_0-9]+)\s*\(',
                       src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_function():
    lib = pm.load_library()
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(_ffi.EXPORTS) == names


def test_struct_sizes():
    assert ctypes.sizeof(_ffi.Plane) == 48
    assert ctypes.sizeof(_ffi.Intrinsics) == 32
    assert ctypes.sizeof(_ffi.RansacParams) == 32
    assert ctypes.sizeof(_ffi.Frame) == 88
    assert ctypes.sizeof(_ffi.RegionPlane) == 56


def test_last_error_initially_empty_or_text():
    assert isinstance(pm.load_library().pm_last_error(), bytes)


def _create(**kw):
    lib = pm.load_library()
    dp = _ffi.DiffusionParams(kw.get('iters', 10), kw.get('lam', 0.2), kw.get('K', 0.02),
                              kw.get('mode', 0), kw.get('ipl', 0), kw.get('tw', 0), kw.get('th', 0))
    rp = _ffi.RansacParams(kw.get('H', 256), kw.get('thr', 0.01), kw.get('mp', 4),
                           kw.get('mi', 100), 0, 20.0)
    mp = _ffi.MiscParams(kw.get('stencil', 0), 0.001)
    h = ctypes.c_void_p()
    st = lib.pm_create(ctypes.byref(dp), ctypes.byref(rp), ctypes.byref(mp), kw.get('w', 64),
                       kw.get('h', 48), kw.get('frames', 1), ctypes.byref(h))
    return st, h


@pytest.mark.parametrize('kw', [dict(lam=0.3), dict(lam=0.0), dict(K=-1.0), dict(mode=2),
                                dict(ipl=9), dict(H=0), dict(H=4096), dict(thr=0.0),
                                dict(mp=0), dict(mp=65), dict(mi=2), dict(stencil=3),
                                dict(w=0), dict(frames=0), dict(frames=2000),
                                dict(iters=-1), dict(tw=129), dict(th=49), dict(tw=-1)])
def test_create_rejects_bad_parameters_before_touching_the_device(kw):
    st, h = _create(**kw)
    assert st == _ffi.PM_ERR_ARG
    assert h.value is None
    assert len(pm.load_library().pm_last_error()) > 0


def test_scratch_bytes_is_monotone():
    a = pm.scratch_bytes(640, 480, 1, 1024, 12)
    b = pm.scratch_bytes(640, 480, 2, 1024, 12)
    c = pm.scratch_bytes(1280, 720, 1, 1024, 12)
    assert 0 < a < b and a < c
    assert pm.scratch_bytes(0, 480, 1, 1024, 12) == -1


def test_region_ransac_rejects_a_null_context():
    lib = pm.load_library()
    out = (_ffi.RegionPlane * 1)()
    st = lib.pm_ransac_regions(None, None, None, None, 64, 48, 1, 64, 0, out, None)
    assert st == _ffi.PM_ERR_ARG


def test_edge_and_region_calls_reject_a_null_context():
    lib = pm.load_library()
    n = ctypes.c_int(0)
    assert lib.pm_canny(None, None, None, 64, 48, 60, 150, None, None) == _ffi.PM_ERR_ARG
    assert lib.pm_segment(None, None, None, 64, 48, 1, 200, None, ctypes.byref(n),
                          None) == _ffi.PM_ERR_ARG


def test_plane_records_read_as_written():
    """The binding reads the pm_plane array a call fills as one structured
    view; every field must come back as the C struct holds it."""
    from paper_2411_01919_b300.pipeline import Planes
    rng = np.random.default_rng(3)
    for n in (0, 1, 7, 12):
        arr = (_ffi.Plane * 12)()
        for i in range(12):
            p = arr[i]
            p.n[0], p.n[1], p.n[2] = rng.normal(size=3)
            p.d = float(rng.normal())
            p.n_inliers = int(rng.integers(0, 1 << 30))
            p.n_refit = int(rng.integers(-5, 1 << 20))
            p.rms = float(np.float32(rng.random()))
            p.hyp_index = int(rng.integers(-1, 2048))
        got = Planes.from_c(arr, n)
        assert got.planes.shape == (n, 4) and got.planes.dtype == np.float64
        for i in range(n):
            p = arr[i]
            assert list(got.planes[i]) == [p.n[0], p.n[1], p.n[2], p.d]
            assert got.n_inliers[i] == p.n_inliers and got.n_refit[i] == p.n_refit
            assert got.rms[i] == np.float32(p.rms) and got.hyp_index[i] == p.hyp_index
