"""Builds libdg.so (the C-ABI library of include/dg.h) in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel to an object file under
``_build/<machine>/``; the objects are linked into
``paper_1601_07944_gb300/libdg.so``, and a stamp beside the objects records
that the library was linked on this machine type.
A unit is recompiled only when it, or a header, is newer than its object.

``build(debug=True)`` makes ``libdg_debug.so`` (objects under
``_build/<machine>-debug/``) with ``-DDG_DEBUG``: every kernel then checks each
connectivity index it reads before using it and reports a bad one through
``dg_device_status`` (a stand-in for a memory checker).
"""
from __future__ import annotations

import glob
import os
import platform
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build", platform.machine())
LIB = os.path.join(PKG, "libdg.so")
LIB_DEBUG = os.path.join(PKG, "libdg_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def build(verbose: bool = False, force: bool = False, debug: bool = False) -> str:
    build_dir = BUILD + "-debug" if debug else BUILD
    lib = LIB_DEBUG if debug else LIB
    flags = ["-DDG_DEBUG"] if debug else []
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    headers = (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
               + glob.glob(os.path.join(ROOT, "include", "*.h")))
    newest_hdr = max((os.path.getmtime(h) for h in headers), default=0.0)
    jobs, objs = [], []
    for src in sources():
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        objs.append(obj)
        if (not force and os.path.exists(obj) and os.path.getmtime(obj) >= os.path.getmtime(src)
                and os.path.getmtime(obj) >= newest_hdr):
            continue
        cmd = [nvcc] + ARCH + COMMON + flags + ["-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        jobs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, pr in jobs:
        out, _ = pr.communicate()
        if pr.returncode != 0:
            failed.append((cmd, out.decode(errors="replace")))
        elif verbose and out:
            sys.stderr.write(out.decode(errors="replace"))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    stamp = os.path.join(build_dir, "libdg.stamp")
    if (force or jobs or not os.path.exists(lib) or not os.path.exists(stamp)
            or any(os.path.getmtime(o) > os.path.getmtime(lib) for o in objs)):
        tmp = lib + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", tmp] + objs)
        os.replace(tmp, lib)
        with open(stamp, "w") as f:
            f.write(lib + "\n")
    return lib


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv, debug="--debug" in sys.argv))
