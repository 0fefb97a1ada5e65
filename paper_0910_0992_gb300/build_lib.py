"""Build libwf.so in-tree with nvcc for sm_103a (GB300).

Usage: ``python paper_0910_0992_gb300/build_lib.py`` (as a script: importing the
package needs the built library) or ``__graft_entry__.build()``.
Each CUDA translation unit is compiled in parallel, then linked into a shared
library next to this file. Object files go to ``_build/`` (git-ignored).
"""

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libwf.so")
SOURCES = ["wf_kernels.cu", "wf_layout.cu", "wf_blas.cu", "wf_abi.cu", "wf_noalloc.cu", "wf_eo4d.cu", "wf_force.cu", "wf_tma.cu", "wf_wide.cu", "wf_wide_df.cu", "wf_pipe.cu", "wf_det.cu", "wf_clover.cu",
           "wf_kernels_long_f32.cu", "wf_kernels_long_f64.cu", "wf_fullsw.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xcompiler", "-Wall", "-Xcompiler", "-Wno-unused-function"]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libwf")
    return path


def _env_flags():
    """Extra nvcc flags from WF_NVCC_FLAGS (tuning sweeps, e.g. -DWF_LINE_MINB=3)."""
    return os.environ.get("WF_NVCC_FLAGS", "").split()


def _compile(src, extra):
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc()] + ARCH + FLAGS + _env_flags() + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(verbose=False, ptxas_info=False):
    """Compile every CUDA source and link libwf.so; returns the library path."""
    os.makedirs(BUILD, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    objs = [o for o, _ in results]
    if verbose or ptxas_info:
        for (_, err), src in zip(results, SOURCES):
            if err.strip():
                print(f"--- {src}\n{err}", file=sys.stderr)
    tmp = LIB + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="-v" in sys.argv))
