"""Compile libminibwa_gpu.so for sm_103a with nvcc (in-tree, under _build/)."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
SO = os.path.join(OUT_DIR, "libminibwa_gpu.so")
PROBE_SRC = os.path.join(HERE, "probe", "gather.cu")
PROBE_SO = os.path.join(OUT_DIR, "libmb_probe.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return "nvcc"


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date() -> bool:
    if not os.path.exists(SO):
        return False
    t = os.path.getmtime(SO)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build_probe(force: bool = False) -> str:
    """The random-gather probe used by bench.py (a separate library, not part of the C ABI)."""
    if not force and os.path.exists(PROBE_SO) and os.path.getmtime(PROBE_SO) >= os.path.getmtime(PROBE_SRC):
        return PROBE_SO
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = PROBE_SO + f".{os.getpid()}.tmp"
    subprocess.check_call([nvcc()] + ARCH + ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                                             PROBE_SRC, "-o", tmp])
    os.replace(tmp, PROBE_SO)
    return PROBE_SO


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    if not force and up_to_date():
        build_probe()
        return SO
    os.makedirs(OUT_DIR, exist_ok=True)
    procs = []
    objs = []
    for src in _sources():
        obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
        objs.append(obj)
        cmd = [nvcc()] + ARCH + FLAGS + (extra or []) + ["-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(cmd)
    if failed:
        raise RuntimeError("nvcc failed: " + " ".join(failed[0]))
    tmp = SO + f".{os.getpid()}.tmp"
    subprocess.check_call([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, SO)
    build_probe(force)
    return SO


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None)
    print(SO)
