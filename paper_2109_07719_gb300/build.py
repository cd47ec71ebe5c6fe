"""Build the CUDA library in-tree: ``csrc/*.cu`` -> ``_lib/libabasim.so``.

Twenty-two translation units (the host side of the C ABI; kernel instantiation
units per precision, direction and adjoint storage mode; the kernels of models
with contact spheres per precision; the world-aligned kernels per precision and
direction, and their pipelined adjoint per precision), compiled by nvcc for sm_103a only, in parallel, then linked; beside it
the FMA-throughput probe ``_lib/fma_peak`` (csrc/fma_peak.cu), an executable that
measures the FP32 and FP64 peaks the roofline fractions divide by.  Called by ``__graft_entry__.build()`` and, lazily, by
the binding when the library is missing or older than its sources.
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libabasim.so")
FMA_PEAK = os.path.join(LIBDIR, "fma_peak")   # the FP32 / FP64 FMA-throughput probe (an executable)
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["abasim.cu", "inst_fp32_fwd.cu", "inst_fp32_bwd.cu", "inst_fp32_bwd_hybrid.cu",
           "inst_fp32_bwd_smem.cu", "inst_mixed_fwd.cu", "inst_mixed_bwd.cu", "inst_mixed_bwd_hybrid.cu",
           "inst_mixed_bwd_smem.cu", "inst_fp64.cu", "inst_fp32_contact.cu", "inst_mixed_contact.cu",
           "inst_fp64_contact.cu", "inst_w_fp32_fwd.cu", "inst_w_fp32_bwd.cu", "inst_w_mixed_fwd.cu", "inst_w_mixed_bwd.cu", "inst_w_fp64_fwd.cu", "inst_w_fp64_bwd.cu", "inst_wp_fp32.cu", "inst_wp_mixed.cu", "inst_wp_fp64.cu"]
DEPS = SOURCES + ["fma_peak.cu", "aba_step.cuh", "contact.cuh", "spatial.cuh", "dual.cuh", "kernels.cuh", "handle.h",
                  "wstep.cuh", "wkernels.cuh", "wpipe.cuh", "tree_order.h"]

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
              "-Xcompiler", "-fPIC", "-diag-suppress", "177"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(FMA_PEAK):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, d) for d in DEPS] + [os.path.join(INCLUDE, "abasim.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the library if it is missing or stale; returns its path."""
    if not force and not stale():
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    tag = f".tmp{os.getpid()}"
    objs = [os.path.join(LIBDIR, os.path.splitext(src)[0] + tag + ".o") for src in SOURCES]

    def compile_one(src_obj):
        src, obj = src_obj
        cmd = [nvcc(), *NVCC_FLAGS, "-I", INCLUDE, "-c", "-o", obj, os.path.join(CSRC, src)]
        if verbose:
            print(" ".join(cmd), flush=True)
        return subprocess.run(cmd, capture_output=True, text=True)

    def compile_tool():
        cmd = [nvcc(), *[f for f in NVCC_FLAGS if f not in ("-Xcompiler", "-fPIC")], "-o", TOOL_TMP,
               os.path.join(CSRC, "fma_peak.cu")]
        return subprocess.run(cmd, capture_output=True, text=True)

    TOOL_TMP = os.path.join(LIBDIR, "fma_peak" + tag)
    with ThreadPoolExecutor(max_workers=len(SOURCES) + 1) as pool:
        tool = pool.submit(compile_tool)
        results = list(pool.map(compile_one, zip(SOURCES, objs)))
        tool = tool.result()
    if tool.returncode != 0:
        raise RuntimeError(f"nvcc failed on fma_peak.cu ({tool.returncode}):\n{tool.stdout}\n{tool.stderr}")
    os.replace(TOOL_TMP, FMA_PEAK)
    for src, r in zip(SOURCES, results):
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src} ({r.returncode}):\n{r.stdout}\n{r.stderr}")
    tmp = os.path.join(LIBDIR, "libabasim" + tag + ".so")
    cmd = [nvcc(), "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    for o in objs:
        if os.path.exists(o):
            os.remove(o)
    if r.returncode != 0:
        raise RuntimeError(f"link failed ({r.returncode}):\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
