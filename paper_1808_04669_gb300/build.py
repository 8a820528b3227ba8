"""Build libdgdf.so in-tree for sm_103a (nvcc + g++, translation units compiled in parallel)."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdgdf.so")

CUDA_SOURCES = ["api.cu", "k_element.cu", "k_stage_df.cu", "k_solver.cu", "k_lattice.cu", "k_multilevel.cu", "k_recover_tc.cu",
                "api3.cu", "k_tet.cu"]
# (source, object name, extra flags): the lattice solver is compiled once per (k, form)
CUDA_VARIANTS = [("k_lattice_inst.cu", "k_lattice_k%d_%d.o" % (k, m), ["-DDG_LAT_K=%d" % k, "-DDG_LAT_MIXED=%d" % m])
                 for k in (1, 2, 3) for m in (0, 1)]
CXX_SOURCES = ["setup.cpp", "host_api.cpp", "multilevel.cpp", "setup3.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _run(cmd):
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError("build step failed: %s\n%s" % (" ".join(cmd), p.stdout))
    return p.stdout


def build(verbose=False, force=False):
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in CUDA_SOURCES + CXX_SOURCES + [v[0] for v in CUDA_VARIANTS]]
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".hpp"))]
    hdrs += [os.path.join(HERE, "..", "include", f) for f in ("dgdf.h", "dgdf_host.h", "dgdf3.h")]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(f) < t for f in srcs + hdrs + [__file__]):
            return LIB
    jobs = []
    for s in CUDA_SOURCES:
        o = os.path.join(BUILD, s + ".o")
        jobs.append([nvcc, "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
                     "-c", os.path.join(CSRC, s), "-o", o])
    for s, oname, flags in CUDA_VARIANTS:
        jobs.append([nvcc, "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", *flags,
                     "-c", os.path.join(CSRC, s), "-o", os.path.join(BUILD, oname)])
    for s in CXX_SOURCES:
        o = os.path.join(BUILD, s + ".o")
        jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-Wall", "-c", os.path.join(CSRC, s), "-o", o])
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    objs = [os.path.join(BUILD, s + ".o") for s in CUDA_SOURCES + CXX_SOURCES]
    objs += [os.path.join(BUILD, v[1]) for v in CUDA_VARIANTS]
    tmp = LIB + ".tmp"
    _run([nvcc, "-shared", *ARCH, "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
