"""The benchmark's reference arm (the CPU oracle, no GPU) prints the one JSON
line the measurement contract asks for: its keys, types and the identities
between them (value, cpu_baseline and e2e describe the same run)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, 'bench.py', '--impl', 'reference', '--steps', '1',
                          '--warmup', '0'], cwd=ROOT, capture_output=True, text=True,
                         timeout=600, check=True).stdout
    lines = [l for l in out.splitlines() if l.startswith('{')]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ('impl', 'metric', 'value', 'unit', 'n_gpus', 'steps', 'warmup', 'ms_per_step',
              'higher_is_better', 'scaling', 'vs_baseline', 'dtype', 'data', 'config',
              'cpu_baseline', 'e2e'):
        assert k in d, k
    assert d['impl'] == 'reference' and d['unit'] == 'frames/s' and d['higher_is_better'] is True
    assert d['steps'] == 1 and d['warmup'] == 0 and d['n_gpus'] == 1
    assert d['value'] > 0 and abs(d['ms_per_step'] - 1e3 / d['value']) < 1e-6 * d['ms_per_step']
    assert d['data'] == 'synthetic' and d['vs_baseline'] is None
    assert 'workload' in d['config']
    # the same workload dict as the GPU arm's line
    sys.path.insert(0, ROOT)
    import bench
    assert d['config'] == bench.shared_config(d['config']['batch_per_gpu'])
    cb = d['cpu_baseline']
    assert cb['kind'] == 'oracle' and cb['cores'] >= 1 and cb['value'] == d['value']
    assert isinstance(cb['sample'], str) and cb['sample']
    e = d['e2e']
    assert e['value'] == d['value'] and e['unit'] == d['unit']
    assert e['h2d_bytes_per_step'] == 0 and e['d2h_bytes_per_step'] == 0
