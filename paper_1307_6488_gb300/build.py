"""Build libbssn.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel; the finite-difference orders
are separate objects of the same source (-DBSSN_ORDER=4/8).
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libbssn.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc")

UNITS = [
    ("bssn_api.cu", "bssn_api.o", []),
    ("bssn_order.cu", "bssn_order4.o", ["-DBSSN_ORDER=4"]),
    ("bssn_order.cu", "bssn_order8.o", ["-DBSSN_ORDER=8"]),
    ("bssn_noalloc.cu", "bssn_noalloc.o", []),
    ("bssn_batch.cu", "bssn_batch.o", []),
    ("bssn_corrector.cu", "bssn_corrector.o", []),
    ("bssn_transfer.cu", "bssn_transfer.o", []),
    ("bssn_amr.cu", "bssn_amr.o", []),
    ("bssn_cfd.cu", "bssn_cfd.o", []),
    ("bssn_checkpoint.cu", "bssn_checkpoint.o", []),
]


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "bssn.h")]


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force=False, verbose=False, ptxas_info=False):
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    flags = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", *ARCH]
    if ptxas_info:
        flags += ["-Xptxas", "-v"]

    def compile_one(unit):
        src, obj, extra = unit
        cmd = [NVCC, "-c", os.path.join(CSRC, src), "-o", os.path.join(BUILD, obj), *flags, *extra]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(compile_one, UNITS))
    for cmd, r in results:
        if verbose or ptxas_info or r.returncode != 0:
            sys.stdout.write(r.stdout)
            sys.stderr.write(r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
    objs = [os.path.join(BUILD, u[1]) for u in UNITS]
    cmd = [NVCC, "-shared", *ARCH, "-o", LIB + ".tmp", *objs]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
