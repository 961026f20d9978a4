"""In-tree build of librom.so for sm_103a (nvcc, one process per translation unit)."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librom.so")
SOURCES = ["api.cu", "fom.cu", "euler.cu", "isvd.cu", "reduced.cu", "sampling.cu", "batch.cu",
           "adjoint.cu", "lspg.cu", "update_rules.cu", "pod_svd.cu"]
# one object per rank bucket and basis type of the iSVD kernels, so that they compile in parallel
BUCKETS = [("isvd_bucket.cu", f"isvd_b{km}_{t}.o",
            [f"-DROM_ISVD_KM={km}", f"-DROM_ISVD_F32={int(t == 'f32')}"])
           for km in (9, 17, 33, 65) for t in ("f64", "f32")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False) -> str:
    """Compile every CUDA translation unit and link librom.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".cuh")]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "rom.h"))
    nvcc = _nvcc()
    units = [(src, src.replace(".cu", ".o"), []) for src in SOURCES] + BUCKETS
    jobs = []
    objs = []
    for src, obj, defs in units:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, obj)
        objs.append(o)
        if _stale(o, [s] + headers):
            jobs.append([nvcc, *ARCH, *FLAGS, *defs, "-c", s, "-o", o])
    # longest first (the widest rank bucket), so the parallel build ends soonest
    jobs.sort(key=lambda cmd: ("-DROM_ISVD_KM=65" not in cmd, "batch.cu" not in cmd[-3]))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))

    with ThreadPoolExecutor(max_workers=max(1, min(len(units), os.cpu_count() or 1))) as ex:
        list(ex.map(run, jobs))
    if jobs or _stale(LIB, objs):
        run([nvcc, *ARCH, "-shared", "-o", LIB, *objs, "-lcudart"])
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
