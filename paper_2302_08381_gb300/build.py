"""Builds libsphericart_gb300.so in-tree with nvcc for sm_103a.

One object per translation unit, compiled in parallel; the POINT kernels are
compiled once per compile-time l_max (``-DSPH_INST_L=<l>``). Objects go to
``_build/`` next to this file and are rebuilt when a source, a header or the
flags change. No CMake, no torch headers.
"""

from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsphericart_gb300.so")
MAX_L_POINT = 16

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _headers_digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            if name.endswith((".h", ".cuh")):
                with open(os.path.join(d, name), "rb") as f:
                    h.update(name.encode() + f.read())
    return h.hexdigest()


def _units():
    units = []
    for l in range(MAX_L_POINT + 1):
        units.append(("sph_point_inst.cu", f"point_L{l}.o", [f"-DSPH_INST_L={l}"]))
    units.append(("sph_degree.cu", "sph_degree_down.o", ["-DSPH_DEGREE_DOWN=1"]))
    for lpp in (1, 2, 4):
        units.append(("sph_degree.cu", f"sph_degree_up{lpp}.o", ["-DSPH_DEGREE_DOWN=0", f"-DSPH_DEGREE_LPP={lpp}"]))
    for part in (0, 1):
        units.append(("sph_row.cu", f"sph_row_{part}.o", [f"-DSPH_ROW_PART={part}"]))
    for gn in range(4):
        units.append(("sph_batch_one.cu", f"sph_batch_one_gn{gn}.o", [f"-DSPH_BATCH_GN={gn}"]))
    for src in ("sph_row_hess.cu", "sph_slice.cu", "sph_capi.cu", "sph_batch.cu", "sph_tune.cu", "sph_expansion.cu", "sph_e3nn.cu", "sph_host.cu", "sph_tables.cpp", "sph_point_registry.cpp"):
        units.append((src, os.path.splitext(src)[0] + ".o", []))
    return units


def _compile(nvcc, src, obj, extra, hdr, verbose):
    path = os.path.join(CSRC, src)
    with open(path, "rb") as f:
        body = f.read()
    cmd = [nvcc] + ARCH + COMMON + extra
    if src.endswith(".cpp"):
        cmd += ["-x", "cu"]
    cmd += ["-c", path, "-o", os.path.join(BUILD, obj)]
    key = hashlib.sha256(body + hdr.encode() + " ".join(cmd).encode()).hexdigest()
    stamp = os.path.join(BUILD, obj + ".key")
    if os.path.exists(os.path.join(BUILD, obj)) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read() == key:
                return obj, False
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src} {extra}:\n{res.stdout}\n{res.stderr}")
    if verbose and res.stderr.strip():
        sys.stderr.write(res.stderr)
    with open(stamp, "w") as f:
        f.write(key)
    return obj, True


def build(verbose: bool = False, jobs: int | None = None) -> str:
    """Compile and link; returns the path of the shared library."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    hdr = _headers_digest()
    units = _units()
    jobs = jobs or max(1, min(len(units), os.cpu_count() or 4))
    changed = False
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        futs = [ex.submit(_compile, nvcc, s, o, e, hdr, verbose) for s, o, e in units]
        for fu in futs:
            _, c = fu.result()
            changed = changed or c
    if changed or not os.path.exists(LIB):
        objs = [os.path.join(BUILD, o) for _, o, _ in units]
        tmp = LIB + ".tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-Xcompiler", "-fPIC", "-o", tmp] + objs
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
