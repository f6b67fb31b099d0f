"""Build libom.so (the CUDA library behind include/om.h) in-tree for sm_103a.

Every .cu file of csrc/ is compiled in parallel with nvcc and linked into
paper_1410_1921_gb300/_build/libom.so against the shared CUDA runtime (the
same libcudart PyTorch loads, so streams and device pointers are shared).
Host code is compiled with -ffp-contract=off: the reconstruction's
acceptance decisions depend on every multiply and add being rounded
separately.
"""
import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libom.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags(verbose=False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                "-I", os.path.join(ROOT, "include")]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _digest(verbose):
    h = hashlib.sha256()
    for p in _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [
            os.path.join(ROOT, "include", "om.h")]:
        h.update(p.encode())
        h.update(open(p, "rb").read())
    h.update(" ".join(_flags(verbose)).encode())
    return h.hexdigest()


def build(force=False, verbose=False, jobs=None):
    """Compile and link; returns the path of libom.so.  Skips work when the
    sources and flags are unchanged since the last build."""
    os.makedirs(OUT, exist_ok=True)
    stamp = os.path.join(OUT, "libom.sha256")
    dig = _digest(verbose)
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    nvcc = _nvcc()
    srcs = _sources()
    objs = [os.path.join(OUT, os.path.basename(s)[:-3] + ".o") for s in srcs]

    def cc(pair):
        s, o = pair
        r = subprocess.run([nvcc] + _flags(verbose) + ["-c", s, "-o", o], capture_output=True, text=True)
        return s, r

    jobs = jobs or min(len(srcs), max(2, os.cpu_count() or 2))
    logs = []
    with cf.ThreadPoolExecutor(jobs) as ex:
        for s, r in ex.map(cc, zip(srcs, objs)):
            logs.append((s, r.stdout + r.stderr))
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {s}:\n{r.stdout}\n{r.stderr}")
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs +
                       ["-Xlinker", "-rpath,/usr/local/cuda/lib64"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    if verbose:
        for s, log in logs:
            print(f"== {os.path.basename(s)}\n{log}")
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
