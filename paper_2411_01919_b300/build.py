"""Build libpm.so (the CUDA kernels and the C ABI) in-tree for sm_103a."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, 'csrc')
LIB = os.path.join(HERE, 'libpm.so')
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
SOURCES = ['pm_api.cu', 'diffuse.cu', 'normals.cu', 'ransac.cu', 'regions.cu', 'canny.cu',
           'noalloc.cu', 'peak.cu', 'map.cpp']


def _nvcc():
    for c in (os.environ.get('NVCC'), '/usr/local/cuda/bin/nvcc', 'nvcc'):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return 'nvcc'


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, '..', 'include', 'pm.h'))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


# the bounds-checking build (PM_DEBUG_BOUNDS): same sources, every instrumented
# kernel access checked against its buffer (see pm_debug_bounds in pm.h)
LIB_BOUNDS = os.path.join(HERE, 'libpm_bounds.so')


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    lib = LIB_BOUNDS if bounds else LIB
    if not force and not _stale(lib):
        return lib
    cmd = [_nvcc(), *ARCH, '-O3', '-lineinfo', '-std=c++17', '-shared', '-Xcompiler', '-fPIC',
           '-Xcompiler', '-Wall', '-o', lib + '.tmp']
    if bounds:
        cmd += ['-DPM_DEBUG_BOUNDS']
    if verbose:
        cmd += ['-Xptxas', '-v']
    cmd += [os.path.join(CSRC, s) for s in SOURCES]
    subprocess.run(cmd, check=True)
    os.replace(lib + '.tmp', lib)
    return lib


if __name__ == '__main__':
    print(build(force='--force' in sys.argv, verbose='-v' in sys.argv,
                bounds='--bounds' in sys.argv))
