"""Build the CUDA library ``liblbmdem.so`` in-tree for sm_103a (GB300).

Each ``csrc/*.cu`` translation unit is compiled in parallel with nvcc, then
linked into ``paper_2003_01490_gb300/_lib/liblbmdem.so``. Usage:
``python -m paper_2003_01490_gb300.build``.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, 'csrc')
OUT_DIR = os.path.join(HERE, '_lib')
OBJ_DIR = os.path.join(HERE, '_build')
LIB = os.path.join(OUT_DIR, 'liblbmdem.so')
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
FLAGS = ['-O3', '-lineinfo', '-std=c++17', '--expt-relaxed-constexpr', '-Xcompiler', '-fPIC',
         '-I' + os.path.join(ROOT, 'include')]


def nvcc():
    for cand in (os.environ.get('NVCC'), shutil.which('nvcc'), '/usr/local/cuda/bin/nvcc'):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError('nvcc not found')


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith('.cu'))


def _compile(args):
    src, obj, extra = args
    cmd = [nvcc(), '-c', src, '-o', obj] + ARCH + FLAGS + extra
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError('nvcc failed for %s:\n%s\n%s' % (src, ' '.join(cmd), r.stderr))
    return r.stderr


def build(verbose=False, extra_flags=()):
    """Compile every translation unit (in parallel) and link the shared library."""
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(OBJ_DIR, exist_ok=True)
    jobs = [(s, os.path.join(OBJ_DIR, os.path.basename(s)[:-3] + '.o'), list(extra_flags))
            for s in sources()]
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(_compile, jobs))
    if verbose:
        for (s, _, _), log in zip(jobs, logs):
            if log.strip():
                print(os.path.basename(s), log)
    tmp = LIB + '.tmp'
    cmd = [nvcc(), '-shared', '-o', tmp] + [j[1] for j in jobs] + ARCH
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError('link failed:\n%s\n%s' % (' '.join(cmd), r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == '__main__':
    extra = sys.argv[1:]
    print(build(verbose=True, extra_flags=extra))
