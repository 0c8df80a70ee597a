"""Builds librte.so (the C-ABI library of include/rte.h) in-tree with nvcc
for sm_103a.  Translation units compile in parallel; the result is
paper_2102_09038_gb300/_build/librte.so."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, 'csrc')
OUT = os.path.join(HERE, '_build')
LIB = os.path.join(OUT, 'librte.so')
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
SOURCES = ['setup_host.cpp', 'mg_host.cpp', 'server.cpp', 'kernels.cu', 'mg.cu', 'tc_gemm.cu',
           'rte.cu', 'dgemm_static.cu', 'tune.cpp', 'e0_direct.cu', 'ec_direct.cu', 'h2.cu',
           'h2_build.cpp']
# host files whose floating point must round the same on every host (no
# contraction into fused multiply-adds)
NO_CONTRACT = ('h2_build.cpp',)


def nvcc():
    cand = shutil.which('nvcc') or '/usr/local/cuda/bin/nvcc'
    if not os.path.exists(cand):
        raise RuntimeError('nvcc not found')
    return cand


def _compile(src, extra):
    obj = os.path.join(OUT, os.path.basename(src) + '.o')
    cmd = [nvcc(), '-O3', '-std=c++17', '-lineinfo', '-Xcompiler', '-fPIC',
           '-I' + os.path.join(HERE, '..', 'include'), '-c', src, '-o', obj]
    cmd += ARCH if src.endswith('.cu') else ['-x', 'c++']
    if os.path.basename(src) in NO_CONTRACT:
        cmd += ['-Xcompiler', '-ffp-contract=off']
    cmd += extra
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError('nvcc failed for %s:\n%s%s' % (src, r.stdout, r.stderr))
    return obj, r.stderr


def _stale(srcs):
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(SRC, f) for f in os.listdir(SRC)]
    deps.append(os.path.join(HERE, '..', 'include', 'rte.h'))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, extra=()):
    """Compile every translation unit and link librte.so; returns its path."""
    os.makedirs(OUT, exist_ok=True)
    srcs = [os.path.join(SRC, s) for s in SOURCES]
    if not force and not _stale(srcs):
        return LIB
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        results = list(ex.map(lambda s: _compile(s, list(extra)), srcs))
    objs = [o for o, _ in results]
    if verbose:
        for _, log in results:
            if log:
                sys.stderr.write(log)
    tmp = LIB + '.tmp'
    cmd = [nvcc(), '-shared', '-o', tmp] + objs + ARCH + [
        '-L/usr/local/cuda/lib64', '-lcusolver', '-lcudart', '-lpthread']
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError('link failed:\n%s%s' % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == '__main__':
    print(build(force='--force' in sys.argv, verbose=True,
                extra=['-Xptxas', '-v'] if '--ptxas' in sys.argv else []))
