#!/usr/bin/env python
"""Benchmark of the per-frame hot path (diffusion -> normals -> RANSAC planes).

Workload: the 640x480 sensor-size staircase (u16 millimetre depth, 6 steps +
floor + landing, sigma = 0.002 z^2, 2% holes + 5-px edge bands; 30 PM4
diffusion iterations, lambda 0.2, K 0.02 m; 1024 hypotheses per plane, 1 cm,
up to 12 planes).  A step is the whole path over one batch of B such frames
(default 64, distinct noise seeds), launched as one graph-captured batch.

Also measured: the plain per-frame path (pm_process_frame, synchronised per
frame), the end-to-end path from pinned host memory, the scoring kernel
against the FP32 roofline, the one-iteration diffusion kernel against HBM,
and the FP64 CPU oracle on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = 'frames/s and p50/p99 frame latency at 640x480, served/batched vs plain; HBM GB/s %'
WORKLOAD = ('640x480 u16 straight staircase (6 steps + floor + landing), 30 PM4 diffusion '
            'iterations, central normals, RANSAC 1024 hypotheses x up to 12 planes, 1 cm')
ITERS, HYP, MAXP, MINI, THR = 30, 1024, 12, 100, 0.01
FP32_FLOP_PER_PAIR = 8          # 3 FMA residual + 1 FMA squared-threshold test
# DRAM bytes (read + write) of the scoring kernel per hypothesis-point pair,
# measured with ncu (dram__bytes_read.sum + dram__bytes_write.sum) on round 0
# of 32 frames of this workload: 155.9 MB for 9.73e9 pairs.  With the number
# of hypotheses fixed, traffic grows with the candidate count, i.e. with pairs.
SCORE_DRAM_BYTES_PER_PAIR = (152.75e6 + 3.11e6) / 9.73e9   # ncu, k_score round 0, 32 frames
SEGMENT, BOX_TEST_FLOP = 32, 14   # box test: 6 FFMA + 2 FADD
N_SETS = 4                      # device copies of the batch the timed steps cycle through


def shared_config(batch):
    """The workload both arms measure (the same dict in both JSON lines);
    what each arm runs it on goes in its own top-level keys."""
    mb = N_SETS * batch * 640 * 480 * 2 / 1e6
    return {'workload': WORKLOAD, 'batch_per_gpu': batch,
            'l2': 'inputs larger than L2: the steps cycle through %d copies of the batch '
                  '(%.0f MB > 126 MB L2)' % (N_SETS, mb),
            'parallelism': 'frames sharded across ranks, no collective (the oracle arm: rank 0 '
                           'alone)'}
REGION_FLOP_PER_PAIR = 9     # 3 FMA residual, |r| x 2^32, 1 FMA inlier test
FP32_LANES = 128              # FP32 lanes per SM (the derived peak printed beside the measured one)


def env_rank():
    return (int(os.environ.get('RANK', 0)), int(os.environ.get('LOCAL_RANK', 0)),
            int(os.environ.get('WORLD_SIZE', 1)))


def peaks():
    p = os.path.join(ROOT, 'MEASURED_PEAKS.json')
    if os.path.exists(p):
        d = json.load(open(p))
        return d, 'measured'
    return {'hbm_gbs': 6400.0, 'sm_max_mhz': 2032.0}, 'fallback'


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
         'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
         'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile('w+', suffix='.csv', delete=False)
        try:
            self.p = subprocess.Popen(['nvidia-smi', '-i', str(index), '--query-gpu=' + self.Q,
                                       '--format=csv,noheader,nounits', '-lms', '50'],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': ['nvidia-smi unavailable']}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(', ') for r in open(self.f.name).read().strip().splitlines() if r]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == 'active':
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {'sm_mhz': statistics.median(sm) if sm else None,
                'sm_max_mhz': max(smax) if smax else None, 'reasons': sorted(reasons),
                'samples': len(sm)}


def make_frames(n, seed0):
    import synth
    return [synth.frame_c2(seed0 + i) for i in range(n)]


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on the same workload
# ---------------------------------------------------------------------------

def oracle_frame_seconds(fr, frame_idx=0):
    import oracle
    t = time.perf_counter()
    oracle.process_frame(fr.encoded, fr.dtype, fr.cam.intrinsics, ITERS, hypotheses=HYP,
                         thr=THR, max_planes=MAXP, min_inliers=MINI, seed=0, frame_idx=frame_idx)
    return time.perf_counter() - t


def diffusion_fused(pipe, B, batch, tuned):
    """The fused (temporally blocked) diffusion of one batch, device-timed:
    its effective rate counts an FP32 iterate read and written per pixel and
    iteration, traffic that shared memory absorbs -- an effective figure, not
    an HBM claim (the kernel is bound by FP32 issue)."""
    pipe.set_timing(1)
    ts = []
    for _ in range(5):
        pipe.process_batch(batch, use_graph=False)
        ts.append(pipe.stage_times()['diffuse_ms'])
    pipe.set_timing(0)
    ms = statistics.median(ts)
    px = sum(int(f['depth'].numel()) for f in batch)
    eff = px * ITERS * 2 * 4 / (ms * 1e-3) / 1e9
    return {'kernel': 'k_diffuse_tiles', 'frames': B, 'iterations': ITERS,
            'tiling': list(tuned['best']) if tuned else 'library default',
            'ms_per_batch': ms, 'effective_gbs': eff,
            'note': 'effective: %d iterations x (4 B read + 4 B written) per pixel, which the '
                    'tiles keep in shared memory; the kernel is FP32-issue bound' % ITERS}


def _oracle_worker(job):
    fr, idx = job
    return oracle_frame_seconds(fr, idx)


def _oracle_ready(_):
    import oracle
    oracle.lib()
    return os.getpid()


def host_cpu_model():
    try:
        with open('/proc/cpuinfo') as fh:
            for line in fh:
                if line.startswith('model name'):
                    return line.split(':', 1)[1].strip()
    except OSError:
        pass
    return 'unknown'


def oracle_all_cores(frames):
    """The oracle on every host core at once: one frame per process (a spawn
    pool, so no child inherits the parent's CUDA context), frames/s from the
    wall time of the whole set."""
    import multiprocessing as mp
    n = max(1, min(os.cpu_count() or 1, 64, len(frames)))
    jobs = [(frames[i], i) for i in range(n)]
    ctx = mp.get_context('spawn')
    with ctx.Pool(n) as pool:
        pool.map(_oracle_ready, range(4 * n))       # start-up outside the timed region
        t = time.perf_counter()
        secs = pool.map(_oracle_worker, jobs, chunksize=1)
        wall = time.perf_counter() - t
    return {'value': n / wall, 'unit': 'frames/s', 'cores': n, 'kind': 'oracle',
            'host': host_cpu_model(),
            'sample': '%d frames of the batch, one single-threaded C oracle process per core, '
                      'wall %.1f s (%.1f-%.1f s per frame)' % (n, wall, min(secs), max(secs))}


def oracle_frame_stages(fr, frame_idx=0):
    """The oracle's frame (the chain oracle.process_frame runs: decode,
    diffusion, normals, RANSAC on the FP32 points), each stage timed."""
    import oracle
    t0 = time.perf_counter()
    zs = oracle.diffuse(oracle.decode(fr.encoded, fr.dtype, 0.001), ITERS)
    t1 = time.perf_counter()
    P, N, V = oracle.normals(zs, fr.cam.intrinsics, 0)
    t2 = time.perf_counter()
    oracle.ransac(P.astype(np.float32), N.astype(np.float32), V, HYP, THR, MAXP, MINI, 0, 20.0,
                  frame_idx)
    t3 = time.perf_counter()
    return t3 - t0, {'decode_diffuse_s': t1 - t0, 'normals_s': t2 - t1, 'ransac_s': t3 - t2}


def run_reference(args):
    rank, _, world = env_rank()
    if rank != 0:
        return 0
    frames = make_frames(max(1, args.warmup + args.steps), 0)
    for i in range(args.warmup):
        oracle_frame_seconds(frames[i], i)
    ts = [oracle_frame_seconds(frames[args.warmup + k], k) for k in range(args.steps)]
    tot = sum(ts)
    value = args.steps / tot
    sample = '1 frame per step (of the %d-frame batch), single-threaded C oracle' % args.batch
    line = {'impl': 'reference', 'metric': METRIC, 'value': value, 'unit': 'frames/s',
            'n_gpus': world, 'steps': args.steps, 'warmup': args.warmup,
            'ms_per_step': 1e3 * tot / args.steps, 'higher_is_better': True, 'scaling': 'weak',
            'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic',
            'config': shared_config(args.batch),
            'form': 'FP64 CPU oracle on one host core; each step times one frame of the batch '
                    '(a bounded sample), frames/s from those frames',
            'cpu_baseline': {'value': value, 'unit': 'frames/s', 'cores': 1, 'kind': 'oracle',
                             'sample': sample},
            'e2e': {'value': value, 'unit': 'frames/s', 'h2d_bytes_per_step': 0,
                    'd2h_bytes_per_step': 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]


def diffusion_hbm(torch, pm, dev, pk, side=8192, iters=10, reps=5, dtype='u16'):
    """Diffusion with one iteration per launch (the streaming kernel, the
    HBM-bound form) on a side x side depth image in the sensor encoding,
    `iters` launches.  Algorithmic bytes (the method's own traffic): per pixel
    and iteration an FP32 iterate read and written (4 + 4 B), plus the first
    read of the encoding (s = 2 B for u16): px (8 N + s).  Moved bytes (what
    the kernels read and write): the first launch reads the encoding and
    writes the lo parts of the compensated iterate (s + 4 B), every later one
    reads the encoding and the lo parts and writes lo parts or, last, FP32
    depth (s + 8 B): px (s + 4 + (N - 1)(s + 8)).  The working set (encoding,
    two lo buffers, output: about 940 MB at 8192^2 u16) is >= 7x L2."""
    s_in = 2 if dtype == 'u16' else 4
    p = pm.Params(iters=iters, iters_per_launch=1)
    pipe = pm.Pipeline(p, side, side, 1)
    g = torch.Generator(device=dev).manual_seed(1)
    zm = 1.0 + 2.0 * torch.rand((side, side), generator=g, device=dev)
    zm[torch.rand((side, side), generator=g, device=dev) < 0.02] = 0.0
    z = ((zm * 1000.0).round().to(torch.int32).to(torch.uint16) if dtype == 'u16'
         else zm.to(torch.float32))
    out = torch.empty((side, side), dtype=torch.float32, device=dev)
    s = torch.cuda.current_stream()
    for _ in range(2):
        pipe.diffuse(z, out)
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        pipe.diffuse(z, out)
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    pipe.close()
    ms = statistics.median(ts)
    px = float(side) * side
    alg = px * (8.0 * iters + s_in)
    moved = px * (s_in + 4.0 + (iters - 1) * (s_in + 8.0))
    gbs = alg / (ms * 1e-3) / 1e9
    mgbs = moved / (ms * 1e-3) / 1e9
    return {'kernel': 'k_diffuse_stream (1 iteration per launch, %d launches)' % iters,
            'image': '%dx%d %s' % (side, side, dtype), 'iterations': iters,
            'algorithmic_bytes_per_call': alg,
            'algorithmic_bytes': 'px x (8 N + %d): FP32 iterate read + written per iteration, '
                                 'encoding read once' % s_in,
            'moved_bytes_per_call': moved,
            'moved_bytes': 'px x (%d + (N - 1) x %d): the encoding re-read by every launch (the '
                           'fixed hi parts), the 4-byte lo parts in and out' % (s_in + 4, s_in + 8),
            'ms': ms, 'achieved': gbs, 'peak': pk['hbm_gbs'], 'unit': 'GB/s',
            'frac': gbs / pk['hbm_gbs'], 'moved_gbs': mgbs, 'moved_frac': mgbs / pk['hbm_gbs']}


def normals_hbm(torch, pm, dev, pk, side=8192, reps=5):
    """Back-projection and normals (pm_normals) on a side x side FP32 depth
    image with 2% holes, outputs preallocated.  Algorithmic bytes per pixel:
    the depth read once (4 B; the stencil's neighbours come from cache) and
    the points, normals and validity written (12 + 12 + 1 B).  The working set
    (about 1.9 GB at 8192^2) is >= 15x L2."""
    g = torch.Generator(device=dev).manual_seed(2)
    z = 1.0 + 2.0 * torch.rand((side, side), generator=g, device=dev)
    z[torch.rand((side, side), generator=g, device=dev) < 0.02] = 0.0
    out = (torch.empty((3, side, side), dtype=torch.float32, device=dev),
           torch.empty((3, side, side), dtype=torch.float32, device=dev),
           torch.empty((side, side), dtype=torch.uint8, device=dev))
    K = (0.6 * side, 0.6 * side, side / 2.0, side / 2.0)
    pipe = pm.Pipeline(pm.Params(iters=1), side, side, 1)
    s = torch.cuda.current_stream()
    for _ in range(2):
        pipe.normals(z, K, out=out)
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        pipe.normals(z, K, out=out)
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    pipe.close()
    ms = statistics.median(ts)
    alg = float(side) * side * 29.0
    gbs = alg / (ms * 1e-3) / 1e9
    return {'kernel': 'k_normals via pm_normals (back-projection, normals, validity)',
            'image': '%dx%d f32' % (side, side), 'algorithmic_bytes_per_call': alg,
            'algorithmic_bytes': 'px x 29: depth read (4 B), points + normals + validity written '
                                 '(12 + 12 + 1 B)',
            'ms': ms, 'achieved': gbs, 'peak': pk['hbm_gbs'], 'unit': 'GB/s',
            'frac': gbs / pk['hbm_gbs']}


def run_regions(torch, pm, pipe, frames, dframes, fp32_peak, n_frames=8, H=256, reps=3):
    """The step after the path, all on the GPU: Canny edges of the normal image,
    the regions they bound, and per-region RANSAC (one model per region) on
    640x480 staircase frames.  Points and normals come from the library's own
    diffusion and normals; the three calls are timed with CUDA events (the
    region count and the planes are read back, so those two synchronise)."""
    s = torch.cuda.current_stream()
    t_edge, t_seg, t_rr, pairs, regions, accepted = [], [], [], 0, 0, 0
    for i in range(n_frames):
        fr = frames[i]
        z = pipe.diffuse(dframes[i])
        P, N, V = pipe.normals(z, fr.cam.intrinsics)
        E = pipe.canny(N, V)                                # warm-up (scratch allocation)
        lab, R = pipe.segment(E, V)
        out = pipe.ransac_regions(P, V, lab, R, H, i)
        for k in range(reps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(s)
            E = pipe.canny(N, V)
            ev[1].record(s)
            lab, R = pipe.segment(E, V)
            ev[2].record(s)
            out = pipe.ransac_regions(P, V, lab, R, H, i)
            ev[3].record(s)
            ev[3].synchronize()
            t_edge.append(ev[0].elapsed_time(ev[1]))
            t_seg.append(ev[1].elapsed_time(ev[2]))
            t_rr.append(ev[2].elapsed_time(ev[3]))
        pairs += int(out.total.sum()) * H
        regions += R
        accepted += int(out.accepted.sum())
    med = statistics.median
    chain = med(t_edge) + med(t_seg) + med(t_rr)
    peak = fp32_peak
    tflops = pairs / n_frames * REGION_FLOP_PER_PAIR / (med(t_rr) * 1e-3) / 1e12
    return {'frames': n_frames, 'regions_per_frame': regions / n_frames,
            'accepted_per_frame': accepted / n_frames, 'hypotheses': H,
            'canny_ms': med(t_edge), 'segment_ms': med(t_seg), 'ransac_regions_ms': med(t_rr),
            'chain_ms_per_frame': chain, 'frames_per_s': 1e3 / chain,
            'regions_per_s': regions / n_frames * 1e3 / med(t_rr),
            'ransac_regions_alu': {'achieved': tflops, 'peak': peak, 'unit': 'TFLOP/s',
                                   'frac': tflops / peak,
                                   'work': '%d FP32 FLOP per hypothesis-point pair, whole call '
                                           '(7 launches)' % REGION_FLOP_PER_PAIR},
            'api': 'pm_canny (60/150) -> pm_segment (gap 1, 200 px) -> pm_ransac_regions, '
                   'one frame per call'}


def run_sweep(torch, pm, pk, frames, dframes, flush):
    """Sec. IV-B's component timing: single-frame time at 320x240 and 640x480
    for 10 / 20 / 40 diffusion iterations (more than 20 for noisier depth),
    both diffusion forms (PM4, Alg. 1 literal) and both normal stencils
    (central, Sobel); the batched 640x480 step with Alg. 1 and with Sobel
    normals (each autotuned); and per-region RANSAC time against the number
    of regions (the paper fits polygons one after another, so its time grows
    linearly with their number)."""
    import synth
    from paper_2411_01919_b300.tune import DiffusionTuner
    s = torch.cuda.current_stream()
    out = {'single_frame': [], 'batched': [], 'regions_vs_count': []}
    for (w, h) in ((320, 240), (640, 480)):
        fr = [synth.frame_straight(sd, w, h) for sd in range(12)]
        dev = [torch.from_numpy(f.encoded).to(dframes[0].device) for f in fr]
        K = fr[0].cam.intrinsics
        for iters in (10, 20, 40):
            for mode in (0, 1):
                for stencil in (0, 1):
                    p = pm.Params(iters=iters, mode=mode, stencil=stencil, hypotheses=HYP, thr=THR,
                                  max_planes=MAXP, min_inliers=MINI, seed=0)
                    with pm.Pipeline(p, w, h, 1) as pipe:
                        for i in range(3):
                            pipe.process_frame(dev[i], K, frame_idx=i, labels=False)
                        ms = []
                        for i in range(len(dev)):
                            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(
                                enable_timing=True)
                            a.record(s)
                            pipe.process_frame(dev[i], K, frame_idx=i, labels=False)
                            b.record(s)
                            b.synchronize()
                            ms.append(a.elapsed_time(b))
                        pipe.set_timing(1)
                        st = []
                        for i in range(6):
                            pipe.process_frame(dev[i], K, frame_idx=i, labels=False)
                            st.append(pipe.stage_times())
                    out['single_frame'].append({
                        'res': '%dx%d' % (w, h), 'iters': iters, 'mode': ['pm4', 'alg1'][mode],
                        'stencil': ['central', 'sobel'][stencil], 'ms_p50': percentile(ms, 50),
                        'diffuse_ms': statistics.median(x['diffuse_ms'] for x in st),
                        'normals_ms': statistics.median(x['normals_ms'] for x in st),
                        'ransac_ms': statistics.median(x['ransac_ms'] for x in st)})
    B = len(frames)
    K = frames[0].cam.intrinsics
    for mode, stencil in ((1, 0), (0, 1)):
        p = pm.Params(iters=ITERS, mode=mode, stencil=stencil, hypotheses=HYP, thr=THR,
                      max_planes=MAXP, min_inliers=MINI, seed=0)
        with pm.Pipeline(p, 640, 480, B) as pipe:
            batch = [dict(depth=dframes[i], K=K, frame_idx=i) for i in range(B)]
            tuned = DiffusionTuner().tune(pipe, batch)
            for _ in range(3):
                pipe.process_batch(batch, use_graph=True)
            ms = []
            for k in range(5):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(s)
                pipe.process_batch(batch, use_graph=True)
                b.record(s)
                b.synchronize()
                ms.append(a.elapsed_time(b))
        out['batched'].append({'mode': ['pm4', 'alg1'][mode], 'stencil': ['central', 'sobel'][stencil],
                               'frames_per_s': B / (statistics.median(ms) * 1e-3),
                               'ms_per_step': statistics.median(ms),
                               'tiling': list(tuned['best'])})
    p = pm.Params(iters=ITERS, hypotheses=HYP, thr=THR, max_planes=MAXP, min_inliers=MINI, seed=0)
    with pm.Pipeline(p, 640, 480, 1) as pipe:
        z = pipe.diffuse(dframes[0])
        P, N, V = pipe.normals(z, K)
        cols = torch.arange(640, device=z.device).view(1, -1).expand(480, 640)
        rows = torch.arange(480, device=z.device).view(-1, 1).expand(480, 640)
        for R in (1, 2, 4, 8, 16, 32, 64, 128):
            gx = int(round(R ** 0.5)) if R > 1 else 1
            while R % gx:
                gx -= 1
            gy = R // gx
            lab = ((rows * gy // 480) * gx + cols * gx // 640).to(torch.int32).contiguous()
            pipe.ransac_regions(P, V, lab, R, 256)
            ms = []
            for k in range(5):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(s)
                pipe.ransac_regions(P, V, lab, R, 256)
                b.record(s)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            out['regions_vs_count'].append({'regions': R, 'hypotheses': 256,
                                            'ms': statistics.median(ms)})
    return out


def _score_rate(torch, pm, pipe, batch, fp32_peak, step_ms):
    """The scoring kernel of one graph-replayed batch: algorithmic work (every
    hypothesis x candidate pair, 8 FLOP) and executed work (evaluated pairs +
    box tests) over its summed launch time, against the measured FP32 peak."""
    pipe.set_timing(2)
    pipe.process_batch(batch, use_graph=True)
    pipe.process_batch(batch, use_graph=True)
    st = pipe.kernel_stats()
    pipe.set_timing(0)
    ms = st['score_ms']
    pairs, ev = st['score_pairs'], st['evaluated_pairs']
    ach = pairs * FP32_FLOP_PER_PAIR / (ms * 1e-3) / 1e12
    exe = (ev * FP32_FLOP_PER_PAIR + pairs / SEGMENT * BOX_TEST_FLOP) / (ms * 1e-3) / 1e12
    return {'kernel': 'k_score', 'achieved': ach, 'frac': ach / fp32_peak, 'executed': exe,
            'executed_frac': exe / fp32_peak, 'evaluated_share': ev / max(1, pairs),
            'kernel_ms_per_step': ms, 'share_of_step': ms / step_ms, 'unit': 'TFLOP/s',
            'peak': fp32_peak}


def run_forms(torch, pm, dev, fp32_peak, flush):
    """The other two configurations the metric's family names, timed on their
    own.  Precision form: 848x480 FP16 spiral staircase (12 steps of 20 deg,
    rise 0.17 m), 40 diffusion iterations, 2048 hypotheses x up to 16 planes;
    16 frames per graph-replayed, autotuned batch, and the plain per-frame
    path.  Batched form: 64 frames of resolutions drawn from {320x240,
    640x480, 848x480, 1280x720}, straight or spiral staircases, FP16 depth,
    20-40 iterations per frame, one graph-replayed autotuned batch per step.
    Each reports frames/s and the scoring kernel's FP32 rates; one precision
    frame's outputs are kept for the per-stage comparison with the oracle."""
    import synth
    from paper_2411_01919_b300.tune import DiffusionTuner
    s = torch.cuda.current_stream()
    workers = min(16, os.cpu_count() or 1)

    def time_batch(pipe, batch, reps=10):
        for _ in range(3):
            pipe.process_batch(batch, use_graph=True)
        ms = []
        for k in range(reps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            pipe.process_batch(batch, use_graph=True)
            b.record(s)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    out = {}
    # precision form
    n3 = 16
    f3 = synth.render_many('frame_c3', [(sd,) for sd in range(n3)], workers)
    d3 = [torch.from_numpy(f.encoded).to(dev) for f in f3]
    p3 = pm.Params(iters=40, hypotheses=2048, max_planes=16, min_inliers=100, seed=5)
    b3 = [dict(depth=d3[i], K=f.cam.intrinsics, frame_idx=i) for i, f in enumerate(f3)]
    with pm.Pipeline(p3, 848, 480, n3) as pipe:
        tuned = DiffusionTuner().tune(pipe, b3)
        ms = time_batch(pipe, b3)
        score = _score_rate(torch, pm, pipe, b3, fp32_peak, ms)
        # one frame's outputs for the per-stage comparison with the oracle
        z = torch.empty((480, 848), dtype=torch.float32, device=dev)
        lab = torch.empty((480, 848), dtype=torch.int16, device=dev)
        one = [dict(depth=d3[1], K=f3[1].cam.intrinsics, frame_idx=1, depth_out=z, labels=lab)]
        pl = pipe.process_batch(one, use_graph=False)[0]
        P, N, V = pipe.frame_geometry(0, 848, 480)
        sample = dict(frame=f3[1], params=p3, frame_idx=1, depth=z.cpu().numpy(),
                      P=P.cpu().numpy(), N=N.cpu().numpy(), V=V.cpu().numpy(), planes=pl,
                      labels=lab.cpu().numpy())
    with pm.Pipeline(p3, 848, 480, 1) as pipe:
        for i in range(3):
            pipe.process_frame(d3[i], f3[i].cam.intrinsics, frame_idx=i, labels=False)
        lat = []
        for i in range(n3):
            t0 = time.perf_counter()
            pipe.process_frame(d3[i], f3[i].cam.intrinsics, frame_idx=i, labels=False)
            lat.append(1e3 * (time.perf_counter() - t0))
        pipe.set_timing(1)
        st = []
        for i in range(6):
            pipe.process_frame(d3[i], f3[i].cam.intrinsics, frame_idx=i, labels=False)
            st.append(pipe.stage_times())
    out['precision_848x480_fp16'] = {
        'batched': {'frames': n3, 'frames_per_s': n3 / (ms * 1e-3), 'ms_per_step': ms,
                    'tiling': list(tuned['best']), 'score': score},
        'plain': {'frames_per_s': len(lat) / (sum(lat) * 1e-3), 'p50_ms': percentile(lat, 50),
                  'p99_ms': percentile(lat, 99),
                  'stage_ms_median': {k: statistics.median(x[k] for x in st) for k in st[0]}},
        'config': '848x480 FP16 spiral, 40 iterations, 2048 hypotheses x 16 planes, 1 cm'}
    out['c3_sample'] = sample
    # batched form, mixed resolutions
    f4 = synth.render_many('frame_c4', [(11, i) for i in range(64)], workers)
    d4 = [torch.from_numpy(f.encoded).to(dev) for f in f4]
    p4 = pm.Params(iters=30, hypotheses=HYP, max_planes=MAXP, min_inliers=MINI, seed=2)
    b4 = [dict(depth=d4[i], K=f.cam.intrinsics, frame_idx=i, iters=f.meta['iters'])
          for i, f in enumerate(f4)]
    with pm.Pipeline(p4, 1280, 720, 64) as pipe:
        tuned4 = DiffusionTuner().tune(pipe, b4)
        ms4 = time_batch(pipe, b4)
        score4 = _score_rate(torch, pm, pipe, b4, fp32_peak, ms4)
    res = {}
    for f in f4:
        k = '%dx%d' % (f.w, f.h)
        res[k] = res.get(k, 0) + 1
    out['batched_mixed_64'] = {
        'frames': 64, 'frames_per_s': 64 / (ms4 * 1e-3), 'ms_per_step': ms4,
        'megapixels_per_s': sum(f.w * f.h for f in f4) / (ms4 * 1e-3) / 1e6,
        'resolutions': res, 'iters': [min(f.meta['iters'] for f in f4),
                                      max(f.meta['iters'] for f in f4)],
        'tiling': list(tuned4['best']), 'score': score4,
        'config': '64 mixed-resolution FP16 frames, 20-40 iterations, 1024 hypotheses x 12 planes'}
    return out


def c3_stage_errors(sample):
    """The precision form's errors against the FP64 oracle, stage by stage on
    one frame, each oracle stage fed the GPU's output of the stage before:
    diffusion (max |z - z_oracle|), points, normals (max angle), and per plane
    the winner, inlier and refit counts, labels, and the plane's angle and
    offset."""
    import oracle
    fr, p = sample['frame'], sample['params']
    f32 = lambda x: float(np.float32(x))
    t0 = time.perf_counter()
    z = oracle.diffuse(oracle.decode(fr.encoded, fr.dtype, f32(p.depth_scale)), p.iters,
                       f32(p.lam), f32(p.K), p.mode)
    dg = sample['depth'].astype(np.float64)
    Po, No, Vo = oracle.normals(dg, fr.cam.intrinsics, p.stencil)
    V = sample['V']
    ok = (V & 2) > 0
    cosang = np.clip(np.abs(np.sum(sample['N'][:, ok].astype(np.float64) * No[:, ok], axis=0)),
                     0.0, 1.0)
    r = oracle.ransac(sample['P'], sample['N'], V, p.hypotheses, p.thr, p.max_planes,
                      p.min_inliers, p.seed, p.gate_deg, sample['frame_idx'])
    g = sample['planes']
    n = min(len(g.planes), len(r.planes))
    angs = [float(np.degrees(np.arccos(min(1.0, abs(float(g.planes[k, :3] @ r.planes[k, :3]))))))
            for k in range(n)]
    offs = [float(abs(g.planes[k, 3] - r.planes[k, 3])) for k in range(n)]
    return {'frame': 'seed 1 of the precision form (848x480 FP16)',
            'diffusion_max_abs_m': float(np.abs(dg - z).max()),
            'diffusion_bar_m': 5e-4,
            'points_max_abs_m': float(np.abs(sample['P'].astype(np.float64) - Po).max()),
            'validity_bits_equal': bool(np.array_equal(V, Vo)),
            'normals_max_deg': float(np.degrees(np.arccos(cosang)).max()) if ok.any() else 0.0,
            'planes': {'gpu': len(g.planes), 'oracle': len(r.planes),
                       'winners_equal': bool(np.array_equal(g.hyp_index, r.hyp_index)),
                       'inlier_counts_equal': bool(np.array_equal(g.n_inliers, r.n_inliers)),
                       'refit_counts_equal': bool(np.array_equal(g.n_refit, r.n_refit)),
                       'labels_equal': bool(np.array_equal(sample['labels'], r.labels)),
                       'max_angle_deg': max(angs) if angs else None,
                       'max_offset_m': max(offs) if offs else None,
                       'near_threshold_band': [int(b) for b in r.band]},
            'oracle_s': time.perf_counter() - t0,
            'method': 'each oracle stage on the GPU output of the stage before (teacher forcing)'}


def run_served(torch, pm, args, c2_frames, c2_dev):
    """The served form: 16 simulated cameras (fixed resolution each from
    424x240 / 640x480 / 848x480 / 1280x720, staircases, camera advancing 5 cm
    per frame), Poisson arrivals with a mean gap of 33 ms, continuous batching
    under a 4 GiB budget, real time for --served-seconds; then the capacity of
    the same loop with every request visible at once, on that stream mix and
    on the 640x480 workload alone; and 16 cameras at 640x480 in real time for
    a third of --served-seconds (at least 5 s)."""
    import synth
    from paper_2411_01919_b300.serve import Request, Server, poisson_arrivals, summarize
    n_streams, poses = 16, 4
    pool = synth.stream_pool(n_streams, poses, seed=0, workers=8)
    host = {s: [torch.from_numpy(np.ascontiguousarray(f.encoded)).pin_memory() for f in fr]
            for s, fr in pool.items()}
    p = pm.Params(iters=30, hypotheses=HYP, thr=THR, max_planes=MAXP, min_inliers=MINI, seed=0)

    def make_reqs(arr):
        return [Request(s, k, t, host[s][k % poses], pool[s][k % poses].cam.intrinsics,
                        frame_idx=k) for s, k, t in arr]

    out = {'streams': n_streams, 'rate_per_stream_hz': 30, 'budget_bytes': 4 << 30,
           'resolutions': sorted({'%dx%d' % (f[0].w, f[0].h) for f in pool.values()}),
           'distinct_poses_per_stream': poses}
    # lanes sized for 1280x720: three of 10 frames hold 2.15 GiB of the 4 GiB
    # budget (two of 16 frames: 2.29 GiB, and less capacity)
    srv = Server(p, budget_bytes=4 << 30, max_batch=10, n_lanes=3)
    srv.run(make_reqs(poisson_arrivals(n_streams, 2.0, 1 / 30, seed=99)))   # warm-up
    arr = poisson_arrivals(n_streams, args.served_seconds, 1 / 30, seed=1)
    reqs = srv.run(make_reqs(arr), realtime=True)
    out.update({'duration_s': args.served_seconds, 'offered': len(arr),
                'offered_frames_per_s': len(arr) / args.served_seconds})
    out['realtime'] = summarize(reqs, srv.elapsed)
    cap = srv.run(make_reqs([(s, k, 0.0) for k in range(40) for s in range(n_streams)]),
                  realtime=False)
    out['capacity_mix'] = summarize(cap, srv.elapsed)
    srv.close()
    # 640x480 only: three lanes of 16 frames hold 1.1 GiB
    srv = Server(p, budget_bytes=4 << 30, max_batch=args.served_batch, n_lanes=3, max_w=640,
                 max_h=480)
    h2 = [torch.from_numpy(f.encoded).pin_memory() for f in c2_frames]
    def c2_reqs():
        return [Request(i % 16, i, 0.0, h2[i % len(h2)], c2_frames[0].cam.intrinsics,
                        frame_idx=i) for i in range(2560)]
    srv.run(c2_reqs()[:128], realtime=False)                                  # warm-up
    # the same 16 cameras at 640x480 in real time (Poisson, 30 Hz each)
    rt_s = max(5.0, args.served_seconds / 3)
    arr2 = poisson_arrivals(n_streams, rt_s, 1 / 30, seed=2)
    rt2 = srv.run([Request(s, k, t, h2[(4 * s + k) % len(h2)], c2_frames[0].cam.intrinsics,
                           frame_idx=k) for s, k, t in arr2], realtime=True)
    out['realtime_640x480'] = dict(summarize(rt2, srv.elapsed), duration_s=rt_s,
                                   offered=len(arr2))
    runs = []
    for _ in range(5):                   # a run of 0.3 s is noisy: the median of five
        cap2 = srv.run(c2_reqs(), realtime=False)
        runs.append(summarize(cap2, srv.elapsed))
    order = sorted(range(5), key=lambda i: runs[i]['frames_per_s'])
    out['capacity_640x480'] = dict(runs[order[2]],
                                   runs_frames_per_s=[r['frames_per_s'] for r in runs])
    srv.close()
    return out


def run_ours(args):
    import torch
    import paper_2411_01919_b300 as pm

    rank, local, world = env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl')
    torch.cuda.set_device(local)
    dev = torch.device('cuda', local)
    pk, pk_kind = peaks()
    meas = pm.measure_peaks()           # FFMA and ex2 throughput of this device, its SM count
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    B = args.batch
    from paper_2411_01919_b300.shard import max_over_ranks, rank_frame_seeds
    frames = [__import__('synth').frame_c2(sd) for sd in rank_frame_seeds(rank, world, B)]
    dframes = [torch.from_numpy(f.encoded).to(dev) for f in frames]
    K = frames[0].cam.intrinsics
    params = pm.Params(iters=ITERS, hypotheses=HYP, thr=THR, max_planes=MAXP, min_inliers=MINI,
                       seed=0)
    pipe = pm.Pipeline(params, 640, 480, B)
    tuned = None
    if args.tiling:
        tuned = {'best': tuple(int(v) for v in args.tiling.split(','))}
        pipe.set_tiling(*tuned['best'])
    elif not args.no_tune:
        from paper_2411_01919_b300.tune import DiffusionTuner
        tuned = DiffusionTuner().tune(pipe, [dict(depth=dframes[i], K=frames[i].cam.intrinsics,
                                                  frame_idx=i) for i in range(B)])
    fused = diffusion_fused(pipe, B, [dict(depth=dframes[i], K=frames[i].cam.intrinsics,
                                            frame_idx=i) for i in range(B)], tuned)
    pipe.set_timing(2)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    s = torch.cuda.current_stream()
    # Whole-job throughput: --lanes pipelines on their own streams take the
    # steps in turn through the asynchronous batch API, so the host prepares
    # and submits the next steps while earlier ones run and their kernels
    # share the GPU.  The steps cycle through
    # N_SETS device copies of the batch (N_SETS x 39 MB > the 126 MB L2), so no
    # step finds its input in L2.
    lanes = [(pipe, torch.cuda.Stream())]
    for _ in range(args.lanes - 1):
        extra = pm.Pipeline(params, 640, 480, B)
        if tuned:
            extra.set_tiling(*tuned['best'])
        extra.set_timing(2)
        lanes.append((extra, torch.cuda.Stream()))
    NL = len(lanes)
    sets = [dframes] + [[d.clone() for d in dframes] for _ in range(N_SETS - 1)]

    def batch(step):
        src = sets[step % N_SETS]
        return [dict(depth=src[i], K=K, frame_idx=step * B + i) for i in range(B)]

    for w in range(args.warmup):
        for lp, ls in lanes:
            with torch.cuda.stream(ls):
                lp.process_batch(batch(w), use_graph=True, stream=ls)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms, score_ms, score_pairs, eval_pairs, launches = [], 0.0, 0, 0, 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    done = [None] * NL
    t_sub = [0.0] * NL

    def finish(li):
        lp, _ = lanes[li]
        nonlocal score_ms, score_pairs, eval_pairs, launches
        done[li].synchronize()
        lp.collect_batch()
        step_ms.append(1e3 * (time.perf_counter() - t_sub[li]))
        st = lp.kernel_stats()
        score_ms += st['score_ms']
        score_pairs += st['score_pairs']
        eval_pairs += st['evaluated_pairs']
        launches += st['launches']
        done[li] = None

    torch.cuda.nvtx.range_push('timed')
    e0.record(s)
    for _, ls in lanes:
        ls.wait_event(e0)
    for k in range(args.steps):
        li = k % NL
        lp, ls = lanes[li]
        if done[li] is not None:
            finish(li)
        t_sub[li] = time.perf_counter()
        with torch.cuda.stream(ls):
            lp.submit_batch(batch(args.warmup + k), use_graph=True, stream=ls)
        ev = torch.cuda.Event()
        ev.record(ls)
        done[li] = ev
    for li in range(NL):
        if done[li] is not None:
            s.wait_event(done[li])
    e1.record(s)
    for li in range(NL):
        if done[li] is not None:
            finish(li)
    e1.synchronize()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    tot_ms = max_over_ranks(e0.elapsed_time(e1), device=dev)
    value = world * B * args.steps / (tot_ms * 1e-3)

    # plain per-frame path: pm_process_frame, synchronised per frame
    pipe1 = pm.Pipeline(params, 640, 480, 1)
    for i in range(3):
        pipe1.process_frame(dframes[i], K, frame_idx=i, labels=False)
    lat = []
    n_plain = min(args.plain_frames, B)
    torch.cuda.nvtx.range_push('plain')
    for i in range(n_plain):
        t0 = time.perf_counter()
        pipe1.process_frame(dframes[i], K, frame_idx=i, labels=False)
        lat.append(1e3 * (time.perf_counter() - t0))
    torch.cuda.nvtx.range_pop()
    pipe1.set_timing(1)
    stage = []
    for i in range(min(8, B)):
        pipe1.process_frame(dframes[i], K, frame_idx=i, labels=False)
        stage.append(pipe1.stage_times())
    plain = {'value': len(lat) / (sum(lat) * 1e-3), 'unit': 'frames/s',
             'p50_ms': percentile(lat, 50), 'p99_ms': percentile(lat, 99), 'frames': len(lat),
             'api': 'pm_process_frame, one stream, synchronised per frame',
             'stage_ms_median': {k: statistics.median(x[k] for x in stage) for k in stage[0]}}
    pipe1.close()

    # end to end through the C ABI with host buffers: every step hands the
    # batch's depth in pinned host memory to pm_process_batch_host_async, which
    # copies each frame to the device on the lane's stream and enqueues the
    # path; the planes come back to the host with pm_batch_collect.  The same
    # lanes take the steps in turn, so one lane's copies overlap the others'
    # batches.
    host = [torch.from_numpy(f.encoded).pin_memory() for f in frames]
    ne = args.steps
    for lp, _ in lanes:
        lp.set_timing(0)
    pend = [None] * NL
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hb = [dict(depth=host[i], K=K, frame_idx=i) for i in range(B)]
    for lp, ls in lanes:                       # warm-up of the host entry's graphs
        with torch.cuda.stream(ls):
            lp.submit_batch_host(hb, use_graph=True, stream=ls)
        ls.synchronize()
        lp.collect_batch()
    torch.cuda.synchronize()
    f0.record(s)
    for _, ls in lanes:
        ls.wait_event(f0)
    for k in range(ne):
        li = k % NL
        lp, ls = lanes[li]
        if pend[li] is not None:
            pend[li].synchronize()
            lp.collect_batch()
        with torch.cuda.stream(ls):
            lp.submit_batch_host(hb, use_graph=True, stream=ls)
        ev = torch.cuda.Event()
        ev.record(ls)
        pend[li] = ev
    for li in range(NL):
        if pend[li] is not None:
            s.wait_event(pend[li])
    f1.record(s)
    for li, (lp, _) in enumerate(lanes):
        if pend[li] is not None:
            pend[li].synchronize()
            lp.collect_batch()
    f1.synchronize()
    h2d = sum(h.numel() * h.element_size() for h in host)
    d2h = B * (64 * 48 + 352)   # planes + per-frame state read back by the call
    e2e = {'value': B * ne / (f0.elapsed_time(f1) * 1e-3), 'unit': 'frames/s',
           'h2d_bytes_per_step': h2d, 'd2h_bytes_per_step': d2h,
           'api': 'pm_process_batch_host_async (pinned host depth, copied by the call) + '
                  'pm_batch_collect per step, %d lanes' % NL}
    # the plain frame end to end: pm_process_frame_host, host depth in, planes out
    pipe1 = pm.Pipeline(params, 640, 480, 1)
    for i in range(3):
        pipe1.process_frame_host(frames[i].encoded, K, frame_idx=i)
    lat_h = []
    for i in range(n_plain):
        t0 = time.perf_counter()
        pipe1.process_frame_host(frames[i].encoded, K, frame_idx=i)
        lat_h.append(1e3 * (time.perf_counter() - t0))
    pipe1.close()
    plain['e2e'] = {'value': len(lat_h) / (sum(lat_h) * 1e-3), 'unit': 'frames/s',
                    'p50_ms': percentile(lat_h, 50), 'p99_ms': percentile(lat_h, 99),
                    'api': 'pm_process_frame_host (host depth in, planes out), synchronised'}

    # roofline: the scoring kernel (FP32 ALU bound).  Algorithmic work = every
    # hypothesis against every candidate, 8 FLOP per pair (3 FFMA for the
    # residual, the test and the count).  Executed work = the pairs the kernel
    # evaluates + one box test per hypothesis and 32-candidate segment
    # (14 FLOP); a box test settles the other pairs of its segment exactly
    # (all outside the threshold, or all inside).
    n_score = args.steps * MAXP
    clock_mhz = pk.get('sm_max_mhz', 2032.0)
    derived_tflops = sm_count * FP32_LANES * 2 * clock_mhz * 1e6 / 1e12
    peak_tflops = meas['fp32_tflops']
    tests = score_pairs / SEGMENT
    flop_exec = eval_pairs * FP32_FLOP_PER_PAIR + tests * BOX_TEST_FLOP
    ach = score_pairs * FP32_FLOP_PER_PAIR / (score_ms * 1e-3) / 1e12 if score_ms > 0 else 0.0
    exe = flop_exec / (score_ms * 1e-3) / 1e12 if score_ms > 0 else 0.0
    roof = {'kernel': 'k_score', 'bound': 'alu', 'achieved': ach, 'peak': peak_tflops,
            'unit': 'TFLOP/s', 'frac': ach / peak_tflops,
            'traffic': (SCORE_DRAM_BYTES_PER_PAIR * score_pairs / n_score
                        if SCORE_DRAM_BYTES_PER_PAIR else None),
            'traffic_note': 'bytes per launch, scaled from an ncu capture of round 0 of 32 frames '
                            'by pairs scored; algorithmic bytes are 16 B per candidate per '
                            'hypothesis block',
            'peak_source': 'measured: pm_measure_peaks, an FFMA-only kernel on all %d SMs timed '
                           'with CUDA events (derived %d SMs x %d lanes x 2 FLOP x %.0f MHz = '
                           '%.1f TFLOP/s)' % (meas['sm_count'], sm_count, FP32_LANES, clock_mhz,
                                              derived_tflops),
            'work': 'algorithmic: %d FLOP per hypothesis-candidate pair, %.3e pairs over %d '
                    'launches (H x M per frame and round)'
                    % (FP32_FLOP_PER_PAIR, score_pairs, n_score),
            'executed': {'achieved': exe, 'frac': exe / peak_tflops,
                         'note': '%d FLOP per evaluated pair + %d FLOP per box test (hypothesis x '
                                 '%d-candidate segment); %.3e of the pairs evaluated (%.1f%%), '
                                 'the rest settled by the box test (segment proven free of '
                                 'inliers, or all inliers)'
                                 % (FP32_FLOP_PER_PAIR, BOX_TEST_FLOP, SEGMENT, eval_pairs,
                                    100.0 * eval_pairs / max(1, score_pairs))},
            'kernel_ms_per_step': score_ms / args.steps,
            'share_of_step': (score_ms / args.steps) / (tot_ms / args.steps) if world == 1 else None}

    hbm = diffusion_hbm(torch, pm, dev, pk) if not args.skip_hbm else None
    hbm_f32 = (diffusion_hbm(torch, pm, dev, pk, dtype='f32', reps=3)
               if not args.skip_hbm else None)
    nrm_hbm = normals_hbm(torch, pm, dev, pk) if not args.skip_hbm else None
    regions = (run_regions(torch, pm, pipe, frames, dframes, peak_tflops)
               if not args.skip_regions else None)
    forms = run_forms(torch, pm, dev, peak_tflops, flush) if not args.skip_forms else None
    sweep = run_sweep(torch, pm, pk, frames, dframes, flush) if not args.skip_sweep else None
    served = run_served(torch, pm, args, frames, dframes) if args.served_seconds > 0 else None

    cpu = cpu_all = None
    if rank == 0 and not args.skip_cpu:
        runs = [oracle_frame_stages(frames[i], i) for i in range(args.cpu_frames)]
        secs = [r[0] for r in runs]
        sec = statistics.median(secs)
        stages = {k: statistics.median(r[1][k] for r in runs) for k in runs[0][1]}
        cpu = {'value': 1.0 / sec, 'unit': 'frames/s', 'cores': 1, 'kind': 'oracle',
               'host': host_cpu_model(), 'stages_s_median': stages,
               'sample': 'median of %d of the %d frames of a step, single-threaded C oracle '
                         '(%.1f-%.1f s per frame)' % (len(secs), B, min(secs), max(secs))}
        cpu_all = oracle_all_cores(frames)
        if forms is not None and forms.get('c3_sample') is not None:
            forms['precision_848x480_fp16']['errors_vs_oracle'] = c3_stage_errors(
                forms['c3_sample'])
    if forms is not None:
        forms.pop('c3_sample', None)

    line = {'metric': METRIC, 'value': value, 'unit': 'frames/s', 'n_gpus': world,
            'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': tot_ms / args.steps,
            'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f32',
            'data': 'synthetic',
            'config': shared_config(B),
            'form': 'batched, CUDA graph; %d lanes take the steps in turn through the '
                    'asynchronous batch API; the batch in %d device copies' % (NL, N_SETS),
            'diffusion_tiling': (dict(zip(('iters_per_launch', 'tile_w', 'tile_h'), tuned['best']))
                                 if tuned else 'library default'),
            'latency_ms': {'p50': percentile(step_ms, 50), 'p99': percentile(step_ms, 99),
                           'note': 'submit to collect of a step (%d steps in flight); a batched '
                                   'frame completes with its step' % NL},
            'plain': plain, 'speedup_vs_plain': value / world / plain['value'],
            'served_capacity_vs_plain': (served['capacity_640x480']['frames_per_s'] / plain['value']
                                         if served else None),
            'served': served, 'regions': regions, 'sweep': sweep,
            'e2e': e2e, 'roofline': roof, 'diffusion_hbm': hbm, 'diffusion_hbm_f32': hbm_f32,
            'normals_hbm': nrm_hbm,
            'diffusion_fused': fused, 'forms': forms,
            'measured_peaks': dict(meas, how='pm_measure_peaks: FFMA-only and ex2-only kernels on '
                                             'every SM, CUDA events, device clocks as found'),
            'cpu_baseline': cpu, 'cpu_baseline_all_cores': cpu_all,
            'gpu_launches': launches, 'clocks': clk,
            'paper_context': '>30 Hz whole pipeline; 7.5 ms/frame; <15 ms at 640x480 with 10 '
                             'diffusion + 10 RANSAC iterations (i9-13900HX + RTX 4060 laptop)'}
    if rank == 0:
        print(json.dumps(line), flush=True)
    pipe.close()
    for lp, _ in lanes[1:]:
        lp.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_case(args):
    """One small workload for a profiler capture (no JSON line): the kernel
    named by --case on the given image / batch, `--steps` calls after
    `--warmup` calls.
      stream-u16 / stream-f32: 8192 x 8192 depth, 4 iterations, one per launch
      normals-f32: pm_normals on an 8192 x 8192 FP32 depth image
      tiles-640x480x64: the fused diffusion of the 64-frame 640x480 batch
      path-640x480x32: the whole path over 32 frames of the 640x480 workload"""
    import torch
    import paper_2411_01919_b300 as pm
    import synth
    dev = torch.device('cuda', 0)
    torch.cuda.set_device(0)
    if args.case == 'normals-f32':
        side = 8192
        g = torch.Generator(device=dev).manual_seed(2)
        z = 1.0 + 2.0 * torch.rand((side, side), generator=g, device=dev)
        z[torch.rand((side, side), generator=g, device=dev) < 0.02] = 0.0
        out = (torch.empty((3, side, side), dtype=torch.float32, device=dev),
               torch.empty((3, side, side), dtype=torch.float32, device=dev),
               torch.empty((side, side), dtype=torch.uint8, device=dev))
        K = (0.6 * side, 0.6 * side, side / 2.0, side / 2.0)
        with pm.Pipeline(pm.Params(iters=1), side, side, 1) as pipe:
            for _ in range(args.warmup + args.steps):
                pipe.normals(z, K, out=out)
            torch.cuda.synchronize()
        return 0
    if args.case.startswith('stream-'):
        side = 8192
        g = torch.Generator(device=dev).manual_seed(1)
        zm = 1.0 + 2.0 * torch.rand((side, side), generator=g, device=dev)
        zm[torch.rand((side, side), generator=g, device=dev) < 0.02] = 0.0
        z = ((zm * 1000.0).round().to(torch.int32).to(torch.uint16) if args.case == 'stream-u16'
             else zm.to(torch.float32))
        out = torch.empty((side, side), dtype=torch.float32, device=dev)
        with pm.Pipeline(pm.Params(iters=4, iters_per_launch=1), side, side, 1) as pipe:
            for _ in range(args.warmup + args.steps):
                pipe.diffuse(z, out)
            torch.cuda.synchronize()
        return 0
    n = 64 if args.case == 'tiles-640x480x64' else 32
    frames = [synth.frame_c2(sd) for sd in range(n)]
    d = [torch.from_numpy(f.encoded).to(dev) for f in frames]
    K = frames[0].cam.intrinsics
    p = pm.Params(iters=ITERS, hypotheses=HYP, thr=THR, max_planes=MAXP, min_inliers=MINI, seed=0)
    with pm.Pipeline(p, 640, 480, n) as pipe:
        if args.tiling:
            pipe.set_tiling(*(int(v) for v in args.tiling.split(',')))
        batch = [dict(depth=d[i], K=K, frame_idx=i) for i in range(n)]
        for _ in range(args.warmup + args.steps):
            pipe.process_batch(batch, use_graph=False)
        torch.cuda.synchronize()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=30)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', choices=['ours', 'reference'], default='ours')
    ap.add_argument('--batch', type=int, default=64)
    ap.add_argument('--plain-frames', type=int, default=32)
    ap.add_argument('--skip-cpu', action='store_true')
    ap.add_argument('--skip-hbm', action='store_true')
    ap.add_argument('--skip-regions', action='store_true')
    ap.add_argument('--skip-sweep', action='store_true')
    ap.add_argument('--skip-forms', action='store_true')
    ap.add_argument('--cpu-frames', type=int, default=5,
                    help='frames of the single-core oracle baseline (the median is reported)')
    ap.add_argument('--lanes', type=int, default=3,
                    help='pipelines taking the timed batches in turn (batches in flight)')
    ap.add_argument('--no-tune', action='store_true')
    ap.add_argument('--tiling', default='',
                    help='diffusion tiling T,tile_w,tile_h instead of autotuning (e.g. 8,80,48)')
    ap.add_argument('--served-seconds', type=float, default=60.0)
    ap.add_argument('--served-batch', type=int, default=16,
                    help='frames per batch of the 640x480 server (three lanes)')
    ap.add_argument('--case', default='',
                    choices=['', 'stream-u16', 'stream-f32', 'normals-f32', 'tiles-640x480x64',
                             'path-640x480x32'],
                    help='run one small workload for a profiler capture instead of the benchmark')
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == 'ours':
        print('note: raising --warmup to 3 (timing rule)', file=sys.stderr)
        args.warmup = 3
    if args.case:
        return run_case(args)
    if args.impl == 'reference':
        return run_reference(args)
    return run_ours(args)


if __name__ == '__main__':
    sys.exit(main())
