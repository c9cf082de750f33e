"""Builds libmcsdp.so in-tree for sm_103a: each CUDA/C++ translation unit is compiled in parallel
with nvcc, then linked into paper_1310_6919_gb300/libmcsdp.so (static CUDA runtime)."""
import hashlib
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmcsdp.so")
STAMP = os.path.join(HERE, "libmcsdp.so.sha256")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU = ["kern_sparse.cu", "kern_scm.cu", "kern_dense.cu", "kern_lsolve.cu", "kern_root.cu", "kern_tc.cu", "mcsdp.cu"]
CPP = ["symbolic.cpp"]


def _nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: libmcsdp needs the CUDA toolkit to build")
    return p


def _sources():
    return [os.path.join(CSRC, f) for f in CU + CPP] + [
        os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))] + [
        os.path.join(HERE, "..", "include", "mcsdp.h")]


COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", CSRC]


def source_hash():
    """SHA-256 over every source file's name and bytes and the compiler flags: the library is
    rebuilt whenever any of them changes (file times are not trusted: copies and checkouts can
    leave a stale library newer than its sources)."""
    h = hashlib.sha256()
    for s in sorted(_sources()):
        h.update(os.path.basename(s).encode())
        with open(s, "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH + COMMON[:-1] + CU + CPP).encode())
    return h.hexdigest()


def up_to_date():
    if not (os.path.exists(LIB) and os.path.exists(STAMP)):
        return False
    with open(STAMP) as f:
        return f.read().strip() == source_hash()


def build(force=False, verbose=False):
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = COMMON
    jobs = []
    for f in CU:
        jobs.append([nvcc] + ARCH + common + ["-c", os.path.join(CSRC, f), "-o",
                                               os.path.join(OUT_DIR, f + ".o")])
    for f in CPP:
        jobs.append([nvcc] + common + ["-x", "c++", "-c", os.path.join(CSRC, f), "-o",
                                       os.path.join(OUT_DIR, f + ".o")])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(OUT_DIR, f + ".o") for f in CU + CPP]
    tmp = LIB + ".tmp"
    run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        f.write(source_hash() + "\n")
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
