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
LIB_CHECK = os.path.join(HERE, "libbssn_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc")

UNITS = [
    ("bssn_api.cu", "bssn_api.o", []),
    ("bssn_order.cu", "bssn_order4.o", ["-DBSSN_ORDER=4"]),
    ("bssn_order.cu", "bssn_order8.o", ["-DBSSN_ORDER=8"]),
    ("bssn_stage32.cu", "bssn_stage32_4.o", ["-DBSSN_ORDER=4"]),
    ("bssn_stage32.cu", "bssn_stage32_8.o", ["-DBSSN_ORDER=8"]),
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


def _stale(lib=None):
    lib = lib or LIB
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force=False, verbose=False, ptxas_info=False, bounds_check=False):
    """Build libbssn.so, or with bounds_check=True its bounds-check variant
    libbssn_check.so (-DBSSN_BOUNDS_CHECK, own object directory)."""
    lib = LIB_CHECK if bounds_check else LIB
    build_dir = BUILD + "_check" if bounds_check else BUILD
    if not force and not _stale(lib):
        return lib
    os.makedirs(build_dir, exist_ok=True)
    flags = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", *ARCH]
    if bounds_check:
        flags.append("-DBSSN_BOUNDS_CHECK")
    if ptxas_info:
        flags += ["-Xptxas", "-v"]

    def compile_one(unit):
        src, obj, extra = unit
        cmd = [NVCC, "-c", os.path.join(CSRC, src), "-o", os.path.join(build_dir, obj), *flags, *extra]
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
    objs = [os.path.join(build_dir, u[1]) for u in UNITS]
    cmd = [NVCC, "-shared", *ARCH, "-o", lib + ".tmp", *objs]
    subprocess.run(cmd, check=True)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
