"""The stage-by-stage parity check itself, on the CPU: it accepts outputs that
are exactly what the oracle computes (run through the spawned worker pool the
GPU tests use), and each planted mistake in the "GPU" side -- a depth off by
2e-5 m, a flipped validity bit, one label changed, a different winning
hypothesis, a plane 2 mm off -- fails it."""
import copy

import numpy as np
import pytest

import oracle
import synth
from paper_2411_01919_b300.pipeline import Params, Planes
from e2e_check import chain_job, check_chain, oracle_chain, run_chains


def f32(x):
    return float(np.float32(x))


@pytest.fixture(scope='module')
def case():
    fr = synth.frame_c1(4)
    p = Params(iters=10, hypotheses=256, max_planes=4, min_inliers=100, seed=9)
    z = oracle.diffuse(oracle.decode(fr.encoded, fr.dtype, f32(p.depth_scale)), p.iters,
                       f32(p.lam), f32(p.K), p.mode).astype(np.float32)
    P, N, V = oracle.normals(z.astype(np.float64), fr.cam.intrinsics, p.stencil)
    P, N = P.astype(np.float32), N.astype(np.float32)
    r = oracle.ransac(P, N, V, p.hypotheses, p.thr, p.max_planes, p.min_inliers, p.seed,
                      p.gate_deg, 5)
    planes = Planes(r.planes.copy(), r.n_inliers.copy(), r.n_refit.copy(), r.rms.copy(),
                    r.hyp_index.copy())
    return fr, p, z, P, N, V, planes, r.labels.copy()


def test_accepts_the_oracles_own_outputs_through_the_pool(case):
    fr, p, z, P, N, V, planes, labels = case
    job = chain_job(fr, p, p.iters, 5, z, P, N, V)
    results = run_chains([job, job])
    assert len(results) == 2
    for res in results:
        assert check_chain(res, planes, labels) == len(planes.planes) >= 2


def test_planted_mistakes_fail(case):
    fr, p, z, P, N, V, planes, labels = case
    res = oracle_chain(chain_job(fr, p, p.iters, 5, z, P, N, V))
    check_chain(res, planes, labels)

    z2 = z.copy()
    z2[z2 > 0] += np.float32(2e-5)
    with pytest.raises(AssertionError):
        check_chain(oracle_chain(chain_job(fr, p, p.iters, 5, z2, P, N, V)), planes, labels)

    V2 = V.copy()
    k = np.flatnonzero((V2 & 2).ravel())[17]
    V2.ravel()[k] &= 1
    with pytest.raises(AssertionError):
        check_chain(oracle_chain(chain_job(fr, p, p.iters, 5, z, P, N, V2)), planes, labels)

    lab2 = labels.copy()
    lab2.ravel()[np.flatnonzero(lab2.ravel() >= 0)[3]] = -1
    with pytest.raises(AssertionError):
        check_chain(res, planes, lab2)

    pl2 = copy.deepcopy(planes)
    pl2.hyp_index[1] += 1
    with pytest.raises(AssertionError):
        check_chain(res, pl2, labels)

    pl3 = copy.deepcopy(planes)
    pl3.planes[1, 3] += 2e-3
    with pytest.raises(AssertionError):
        check_chain(res, pl3, labels)


def test_structural_check_accepts_another_draw_and_rejects_wrong_structure():
    """check_end_to_end (the extra, structural comparison) passes two oracle
    runs whose draws differ, and fails a labelling that merges two surfaces
    or misses one."""
    from e2e_check import check_end_to_end
    fr = synth.frame_c1(0)
    runs = [oracle.process_frame(fr.encoded, fr.dtype, fr.cam.intrinsics, 10, f32(0.2),
                                 f32(0.02), hypotheses=256, max_planes=4, min_inliers=100,
                                 seed=s, frame_idx=0, depth_scale=f32(0.001)).ransac
            for s in (11, 12)]
    a, b = runs
    assert not np.array_equal(a.hyp_index, b.hyp_index)
    pb = Planes(b.planes, b.n_inliers, b.n_refit, b.rms, b.hyp_index)
    assert check_end_to_end(fr, pb, b.labels, a, min_big=300) >= 0.9
    # the pixels of the second plane relabelled as the first: two surfaces merged
    merged = b.labels.copy()
    merged[merged == 1] = 0
    with pytest.raises(AssertionError):
        check_end_to_end(fr, pb, merged, a, min_big=300)
    # the second plane missing altogether
    pmiss = Planes(b.planes[[0, 2, 3]], b.n_inliers[[0, 2, 3]], b.n_refit[[0, 2, 3]],
                   b.rms[[0, 2, 3]], b.hyp_index[[0, 2, 3]])
    missing = b.labels.copy()
    missing[missing == 1] = -1
    missing[missing >= 2] -= 1
    with pytest.raises(AssertionError):
        check_end_to_end(fr, pmiss, missing, a, min_big=300)
