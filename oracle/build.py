"""Compile the C oracle into oracle/liboracle.so (test infrastructure only)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, 'oracle.c')
LIB = os.path.join(HERE, 'liboracle.so')


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    # -ffp-contract=off: no implicit FMA, so the FP32 decisions are exactly the
    # operations written in oracle.c.
    cmd = ['gcc', '-O2', '-std=gnu11', '-fPIC', '-shared', '-ffp-contract=off',
           '-fno-fast-math', '-Wall', '-o', LIB + '.tmp', SRC, '-lm']
    subprocess.run(cmd, check=True)
    os.replace(LIB + '.tmp', LIB)
    return LIB


if __name__ == '__main__':
    print(build(force='--force' in sys.argv))
