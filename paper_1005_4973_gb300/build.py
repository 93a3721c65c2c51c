"""Builds libmtgp.so in-tree for sm_103a with nvcc (no cmake, no torch).

    python -m paper_1005_4973_gb300.build [--verbose-ptxas]

The kernel and host translation units compile in parallel, then link into
paper_1005_4973_gb300/_build/libmtgp.so.
"""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libmtgp.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
SOURCES = ["mtgp_kernels.cu", "mtgp_gen_t32.cu", "mtgp_gen_t64.cu", "mtgp_gen_t128.cu", "mtgp_gen_t256.cu",
           "mtgp_gen_t512.cu", "mtgp_split_rt64.cu", "mtgp_split_rt128.cu", "mtgp_split_rt256.cu",
           "mtgp_split_rt512.cu", "mtgp_flow_w2.cu", "mtgp_flow_w4.cu", "mtgp_flow_w8.cu",
           "mtgp_flow_w16.cu", "mtgp_wide.cu", "mtgp_pairs_t128_q2.cu", "mtgp_pairs_t128_q3.cu", "mtgp_pairs_t128_q6.cu", "mtgp_dual_t128_q3.cu", "mtgp_noalloc.cu", "mtgp_jump.cu", "mtgp_bm.cu", "mtgp_irr.cu", "mtgp_host.cpp", "mtgp_jump_host.cpp",
           "mtgp_f2.cpp", "mtgp_search.cpp", "mtgp_equid.cpp",
           "mtgp_server.cpp"]


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "mtgp.h"))
    return files


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, ptxas_verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2",
              "-I", os.path.join(ROOT, "include"), "-I", CSRC] + ARCH
    if ptxas_verbose:
        common += ["-Xptxas", "-v"]
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(OUT_DIR, src + ".o")
        objs.append(obj)
        cmd = [NVCC, "-c", os.path.join(CSRC, src), "-o", obj] + common
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{text}")
        if ptxas_verbose and text.strip():
            sys.stdout.write(text)
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call([NVCC, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart_static", "-lrt", "-lpthread", "-ldl"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, ptxas_verbose="--verbose-ptxas" in sys.argv))
