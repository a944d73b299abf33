"""Build liblmf.so (the C-ABI engine) in-tree with nvcc for sm_103a.

Translation units are compiled in parallel and linked into
paper_1906_08687_gb300/_build/liblmf.so.  Nothing is installed elsewhere.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, 'csrc')
INCLUDE = os.path.join(ROOT, 'include')
OUT_DIR = os.path.join(HERE, '_build')
LIB = os.path.join(OUT_DIR, 'liblmf.so')

ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
FLAGS = ['-O3', '-lineinfo', '-std=c++17', '-Xcompiler', '-fPIC', '--expt-relaxed-constexpr',
         '-I', INCLUDE, '-I', CSRC, '-I', OUT_DIR]
# device headers the plan-time compiler (NVRTC) gets as in-memory sources
JIT_HEADERS = ['lmf_internal.h', 'lmf_rowpass.cuh', 'lmf_root_plain.cuh', 'lmf_root_tc.cuh', 'lmf_root_lean.cuh',
               'lmf_tree_dev.cuh']
JIT_INC = os.path.join(OUT_DIR, 'lmf_jit_headers.inc')


def _nvcc() -> str:
    for cand in (os.environ.get('NVCC'), '/usr/local/cuda/bin/nvcc', 'nvcc'):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return 'nvcc'


def _deps_mtime() -> float:
    files = glob.glob(os.path.join(CSRC, '*')) + glob.glob(os.path.join(INCLUDE, '*.h'))
    return max(os.path.getmtime(f) for f in files)


def write_jit_headers() -> None:
    """Embed the device headers as raw string literals for lmf_jit.cu."""
    names, texts = [], []
    for h in JIT_HEADERS:
        with open(os.path.join(CSRC, h)) as f:
            t = f.read()
        if ')LMFJIT"' in t:
            raise RuntimeError(f'{h} contains the raw-string delimiter')
        names.append(f'"{h}"')
        texts.append('R"LMFJIT(' + t + ')LMFJIT"')
    body = ('// generated by build.py from ' + ', '.join(JIT_HEADERS) + '\n'
            'static const char* const kJitHeaderNames[] = {' + ', '.join(names) + '};\n'
            'static const char* const kJitHeaderSrc[] = {\n' + ',\n'.join(texts) + '};\n')
    old = open(JIT_INC).read() if os.path.exists(JIT_INC) else None
    if old != body:
        with open(JIT_INC, 'w') as f:
            f.write(body)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, '*.cu')))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    write_jit_headers()
    nvcc = _nvcc()

    def compile_one(src: str) -> str:
        obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + '.o')
        cmd = [nvcc] + ARCH + FLAGS + ['-c', src, '-o', obj]
        if verbose:
            print(' '.join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f'nvcc failed on {os.path.basename(src)}:\n{r.stderr}')
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + f'.{os.getpid()}.tmp'
    cmd = [nvcc] + ARCH + ['-shared', '-o', tmp] + objs + ['-ldl']
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f'link failed:\n{r.stderr}')
    os.replace(tmp, LIB)
    return LIB


if __name__ == '__main__':
    print(build(force='--force' in sys.argv, verbose=True))
