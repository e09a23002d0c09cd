"""Builds libcpra.so (the C-ABI library) in-tree for sm_103a with nvcc.

Each translation unit under csrc/ is compiled in parallel, then linked into
``paper_2402_02190_gb300/lib/libcpra.so``.  The checked build,
``lib/libcpra_checked.so``, links the same objects except the translation
units that walk the CSR, which are compiled again with ``-DCPRA_CHECKED``
(in-kernel row-range and column-index checks, see cpra_csr_check).
Objects are rebuilt only when a source or header is newer than the object.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libcpra.so")
LIB_CHECKED = os.path.join(LIBDIR, "libcpra_checked.so")
# the translation units whose kernels read the CSR (and the ABI layer that
# collects their check words)
CHECKED_SRCS = ("cpra_api.cu", "k_eval.cu", "k_loss_problem.cu", "k_spmm.cu")
# sources compiled more than once, each object with its own defines
MULTI = {
    "k_loss_problem.cu": [(f"k_loss_p{p}", [f"-DCPRA_LOSS_PROBLEM={p}"]) for p in range(5)],
    "k_gemm_simt.cu": [(f"k_gemm_simt_{a}{b}", [f"-DCPRA_SIMT_DA={a}", f"-DCPRA_SIMT_DB={b}"])
                       for a in (0, 1) for b in (0, 1)],
}
SLOW_STEMS = ("k_gemm_simt", "k_loss_p", "k_spmm", "k_gemm_tc")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--compress-mode=size", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden", "--expt-relaxed-constexpr",
              "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return hs


def _units():
    """(source, object stem, defines) of every object of the library."""
    out = []
    for src in _sources():
        for stem, defs in MULTI.get(src, [(src[:-3], [])]):
            out.append((src, stem, defs))
    return out


def _compile(nvcc, src, extra, outdir=BUILD, stem=None):
    obj = os.path.join(outdir, (stem or src[:-3]) + ".o")
    srcp = os.path.join(CSRC, src)
    newest = max([os.path.getmtime(srcp)] + [os.path.getmtime(h) for h in _headers()])
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest:
        return obj, ""
    cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", srcp, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stdout + r.stderr


def _link(nvcc, objs, lib):
    newest_obj = max(os.path.getmtime(o) for o in objs)
    if not os.path.exists(lib) or os.path.getmtime(lib) < newest_obj:
        cmd = [nvcc, *ARCH, "-shared", "-o", lib + ".tmp", *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(lib + ".tmp", lib)


def build(verbose: bool = False, extra_flags=None, checked: bool = True) -> str:
    """Compile every csrc/*.cu for sm_103a and link libcpra.so (and, with
    checked=True, libcpra_checked.so); returns the path of libcpra.so."""
    nvcc = _nvcc()
    checked_dir = os.path.join(BUILD, "checked")
    os.makedirs(checked_dir, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    extra = list(extra_flags or [])
    units = _units()
    jobs = [(src, extra + defs, BUILD, stem) for src, stem, defs in units]
    if checked:
        jobs += [(src, extra + defs + ["-DCPRA_CHECKED"], checked_dir, stem)
                 for src, stem, defs in units if src in CHECKED_SRCS]
    # the slowest translation units (the template-heavy kernels) start first
    jobs.sort(key=lambda j: not j[3].startswith(SLOW_STEMS))
    with cf.ThreadPoolExecutor(max_workers=min(os.cpu_count() or 8, len(jobs))) as ex:
        results = list(ex.map(lambda j: _compile(nvcc, *j), jobs))
    if verbose:
        for _, log in results:
            if log.strip():
                print(log)
    objs = [os.path.join(BUILD, stem + ".o") for _, stem, _ in units]
    _link(nvcc, objs, LIB)
    if checked:
        cobjs = [os.path.join(checked_dir if src in CHECKED_SRCS else BUILD, stem + ".o")
                 for src, stem, _ in units]
        _link(nvcc, cobjs, LIB_CHECKED)
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(verbose=v or bool(extra), extra_flags=extra))
