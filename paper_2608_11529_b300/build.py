"""Build the in-tree shared library libe2.so for sm_103a with nvcc."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libe2.so")
SOURCES = ["e2_kernels.cu", "e2_adjoint.cu", "e2_ozaki.cu", "e2_plan.cu", "e2_api.cu", "e2_batch.cu", "e2_grad.cu", "e2_solver.cu"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-shared", "-cudart", "static", "-Xcompiler", "-fvisibility=hidden"]


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "e2.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Compile every source to an object in parallel (one nvcc per unit), then
    link the shared library."""
    if not force and not _stale():
        return LIB
    import concurrent.futures as cf
    import tempfile
    tmp = LIB + f".tmp{os.getpid()}"
    inc = ["-I", os.path.join(ROOT, "include")]
    compile_flags = [f for f in FLAGS if f not in ("-shared", "-cudart", "static")]
    with tempfile.TemporaryDirectory() as td:
        objs = [os.path.join(td, s.replace(".cu", ".o")) for s in SOURCES]
        cmds = [[NVCC, *compile_flags, *inc, "-c", os.path.join(CSRC, s), "-o", o] for s, o in zip(SOURCES, objs)]
        if verbose:
            for c in cmds:
                print(" ".join(c))
        with cf.ThreadPoolExecutor(max_workers=min(len(cmds), os.cpu_count() or 1)) as ex:
            for f in [ex.submit(subprocess.check_call, c) for c in cmds]:
                f.result()
        link = [NVCC, *FLAGS, "-o", tmp] + objs
        if verbose:
            print(" ".join(link))
        subprocess.check_call(link)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
