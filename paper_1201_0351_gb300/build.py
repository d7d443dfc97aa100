"""Builds libgb300_lbmfs.so (sm_103a) in-tree with nvcc.

The translation units compile in parallel: the host API, the batched form,
one kernel unit per population storage, the allocation-free reduction
and the measurement helper.  The double-precision unit is compiled with
-fmad=false (no fused multiply-add) so that it rounds every operation exactly
as the plain CPU restatement of the method does.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libgb300_lbmfs.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
UNITS = {
    "lbmfs_api.cu": [],
    "lbmfs_batch.cu": [],
    "kernels_f64.cu": ["-fmad=false"],
    "kernels_f32.cu": [],
    "kernels_f16s.cu": [],
    "lbmfs_noalloc.cu": [],
    "lbmfs_probe.cu": [],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "lbm_fs.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False, extra_flags=(), out_dir: str = OUT_DIR,
          csrc: str = CSRC) -> str:
    """Compile the library if any source is newer than it; returns its path.
    extra_flags / out_dir / csrc build a variant elsewhere (tuning experiments)."""
    lib = os.path.join(out_dir, os.path.basename(LIB))
    if not force and out_dir == OUT_DIR and csrc == CSRC and not extra_flags and up_to_date():
        return LIB
    os.makedirs(out_dir, exist_ok=True)
    nv = nvcc()
    objs = []
    cmds = []
    for unit, flags in UNITS.items():
        obj = os.path.join(out_dir, unit.replace(".cu", ".o"))
        objs.append(obj)
        cmds.append([nv, *ARCH, "-I", csrc, *COMMON, *flags, *extra_flags, "-c", os.path.join(csrc, unit), "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        for out in ex.map(run, cmds):
            if verbose and out.strip():
                print(out)
    tmp = lib + ".%d.tmp" % os.getpid()
    run([nv, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose=True))
