"""Build the in-tree shared libraries for sm_103a (GB300).

  paper_1908_09606_gb300/_build/libcosma_gb300.so   the C-ABI library (include/cosma.h)
  cosma_inputs/_build/libcosma_inputs.so            the device half of the input generator

Each translation unit is compiled by its own nvcc process (in parallel) and the
objects are linked into one shared object.  Rebuilds only what changed.
"""

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]

LIB = os.path.join(HERE, "_build", "libcosma_gb300.so")
INPUTS_LIB = os.path.join(ROOT, "cosma_inputs", "_build", "libcosma_inputs.so")


def _newer(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, obj, deps, extra=()):
    if not _newer(obj, [src] + deps):
        return obj
    cmd = [NVCC] + ARCH + COMMON + list(extra) + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj


def _link(objs, out, libs=()):
    if not _newer(out, objs):
        return out
    cmd = [NVCC] + ARCH + ["-shared", "-o", out + ".tmp"] + objs + list(libs)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed for {out}:\n{r.stdout}\n{r.stderr}")
    os.replace(out + ".tmp", out)
    return out


def build(verbose=False, jobs=None):
    csrc = os.path.join(HERE, "csrc")
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    headers = glob.glob(os.path.join(csrc, "*.h")) + glob.glob(os.path.join(csrc, "*.cuh")) + \
        [os.path.join(ROOT, "include", "cosma.h")]
    srcs = sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cpp")))
    ibdir = os.path.join(ROOT, "cosma_inputs", "_build")
    os.makedirs(ibdir, exist_ok=True)
    isrc = os.path.join(ROOT, "cosma_inputs", "csrc", "philox_fill.cu")
    jobs = jobs or min(16, (os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(jobs) as ex:
        futs = {}
        for s in srcs:
            obj = os.path.join(bdir, os.path.basename(s) + ".o")
            futs[ex.submit(_compile, s, obj, headers, ["-I", os.path.join(ROOT, "include")])] = s
        ifut = ex.submit(_compile, isrc, os.path.join(ibdir, "philox_fill.o"), [])
        objs = [f.result() for f in futs]
        iobj = ifut.result()
    _link(sorted(objs), LIB)
    _link([iobj], INPUTS_LIB)
    if verbose:
        print("built", LIB, INPUTS_LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
