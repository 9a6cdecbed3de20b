"""Build libkstap.so (sm_103a) in-tree with nvcc.

The library is compiled as several translation units in parallel: the host
logic (csrc/kstap_api.cu) and one unit per class (p, q) and part (fit or
detect) of csrc/kstap_inst.cu, then linked into one shared object.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libkstap.so")
DEPS = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
    os.path.join(os.path.dirname(HERE), "include", "kstap.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17"] + ARCH + ["-lineinfo", "-Xcompiler", "-fPIC",
                                             "-diag-suppress", "177"]
# (p, q) classes with their own translation units; must match KSTAP_CLASSES in
# csrc/kstap_host.cuh
CLASSES = [(3, 8), (3, 12), (3, 16), (3, 24), (3, 32), (6, 8), (6, 16)]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def units():
    """(object name, source, extra defines) of every translation unit."""
    out = [("kstap_api.o", os.path.join(CSRC, "kstap_api.cu"), []),
           ("kstap_peaks.o", os.path.join(CSRC, "kstap_peaks.cu"), [])]
    for p, q in CLASSES:
        for part, name in ((0, "fit"), (1, "detect")):
            out.append((f"kstap_{name}_p{p}_q{q}.o", os.path.join(CSRC, "kstap_inst.cu"),
                        [f"-DKSTAP_INST_P={p}", f"-DKSTAP_INST_Q={q}",
                         f"-DKSTAP_INST_PART={part}"]))
    return out


def build(force: bool = False, verbose: bool = False, jobs: int = 0) -> str:
    newest = max(os.path.getmtime(p) for p in DEPS if os.path.exists(p))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    os.makedirs(OBJ_DIR, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose else []

    def compile_one(u):
        name, src, defs = u
        obj = os.path.join(OBJ_DIR, name)
        if not force and os.path.exists(obj) and os.path.getmtime(obj) >= newest:
            return obj
        tmp = obj + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc()] + NVCC_FLAGS + extra + defs + ["-c", "-o", tmp, src])
        os.replace(tmp, obj)
        return obj

    n = jobs or max(1, min(len(units()), os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=n) as ex:
        objs = list(ex.map(compile_one, units()))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
