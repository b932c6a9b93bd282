"""pm_diffuse_noalloc: diffusion for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc at all -- a hard real-time control loop,
where cudaMalloc/cudaFree can stall the whole device for an unbounded time, or
a plug-in inside a host framework whose own allocator owns the device memory.
For them libpm offers one entry point that needs no context and allocates
nothing: its working iterate lives in a fixed device array inside the library.
These tests call it through the C ABI and compare its output with the regular
pm_diffuse on two calls in a row (the second call reuses the array the first
one left behind), with the FP64 oracle on ragged shapes, zero iterations and
a padded row pitch, and check that an oversize image is refused.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2411_01919_b300 import Params, Pipeline, _ffi

pytestmark = pytest.mark.gpu

DIFF_TOL = 1e-5          # the diffusion tolerance of the other parity tests
CODES = {'u16': _ffi.PM_U16_MM, 'f16': _ffi.PM_F16_M, 'f32': _ffi.PM_F32_M}


def noalloc_diffuse(depth: torch.Tensor, dtype: str, p: Params, out: torch.Tensor) -> int:
    lib = _ffi.load()
    dp = _ffi.DiffusionParams(p.iters, p.lam, p.K, p.mode, 0, 0, 0)
    h, w = depth.shape
    pitch = depth.stride(0) * depth.element_size()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.pm_diffuse_noalloc(ctypes.c_void_p(depth.data_ptr()), CODES[dtype], w, h, pitch,
                                  ctypes.byref(dp), p.depth_scale,
                                  ctypes.c_void_p(out.data_ptr()), stream)


def test_noalloc_matches_pm_diffuse_on_two_calls_in_a_row():
    # a larger frame first, then a smaller one, so stale iterate data from
    # the first call sits in the shared array when the second one runs
    cases = [(synth.frame_c3(2), Params(iters=40)), (synth.frame_c2(7), Params(iters=30)),
             (synth.frame_c1(3), Params(iters=10, mode=1))]
    for fr, p in cases:
        d = torch.from_numpy(fr.encoded).cuda()
        with Pipeline(p, fr.w, fr.h) as pipe:
            ref = pipe.diffuse(d).clone()
        out = torch.full((fr.h, fr.w), -1.0, dtype=torch.float32, device='cuda')
        _ffi.check(noalloc_diffuse(d, fr.dtype, p, out))
        torch.cuda.synchronize()
        err = (out.double() - ref.double()).abs().max().item()
        assert err <= DIFF_TOL, (fr.meta, err)
        assert torch.equal(out == 0, ref == 0)


def ragged_depth(seed, h, w, dtype):
    """A tilted plane with bumps and 3% holes in the given sensor encoding."""
    rng = np.random.default_rng(seed)
    v, u = np.mgrid[0:h, 0:w]
    z = 1.2 + 0.004 * u + 0.002 * v + 0.01 * np.sin(u / 3.0) + rng.normal(0, 0.003, (h, w))
    z[rng.random((h, w)) < 0.03] = 0.0
    if dtype == 'u16':
        return np.round(z * 1000.0).astype(np.uint16)
    if dtype == 'f16':
        return z.astype(np.float16)
    return z.astype(np.float32)


@pytest.mark.parametrize('h,w,dtype,iters,mode,pad', [
    (37, 53, 'u16', 0, 0, 0),      # zero iterations: decode only
    (61, 97, 'u16', 7, 1, 13),     # Alg. 1 form, u16 rows inside a wider buffer
    (45, 33, 'f16', 9, 1, 0),      # Alg. 1 form on FP16 storage
    (130, 257, 'f32', 12, 0, 3),   # odd width, padded pitch
    (1, 300, 'u16', 4, 0, 0),      # a single row
])
def test_noalloc_matches_the_oracle(h, w, dtype, iters, mode, pad):
    enc = ragged_depth(h * 1000 + w, h, w, dtype)
    p = Params(iters=iters, mode=mode)
    wide = np.zeros((h, w + pad), dtype=enc.dtype)
    wide[:, :w] = enc
    d = torch.from_numpy(wide).cuda()[:, :w]          # pitch = (w + pad) * element size
    f32 = lambda x: float(np.float32(x))
    ref = oracle.diffuse(oracle.decode(enc, dtype, f32(p.depth_scale)), iters, f32(p.lam),
                         f32(p.K), mode)
    for _ in range(2):                                  # two calls in a row
        out = torch.full((h, w), -1.0, dtype=torch.float32, device='cuda')
        _ffi.check(noalloc_diffuse(d, dtype, p, out))
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        assert np.abs(got - ref).max() <= DIFF_TOL
        assert np.array_equal(got == 0, ref == 0)
    with Pipeline(p, w, h) as pipe:
        assert torch.equal(pipe.diffuse(d), out)


def test_noalloc_refuses_images_above_its_limit():
    p = Params(iters=2)
    side = int(np.ceil(np.sqrt(_ffi.PM_NOALLOC_MAX_PIXELS))) + 1
    d = torch.ones((side, side), dtype=torch.float32, device='cuda')
    out = torch.empty_like(d)
    st = noalloc_diffuse(d, 'f32', p, out)
    assert st == _ffi.PM_ERR_ARG
    assert b'PM_NOALLOC_MAX_PIXELS' in _ffi.load().pm_last_error()
