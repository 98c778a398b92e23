"""Build libpdg.so in-tree with nvcc for sm_103a (GB300).

The translation units are compiled in parallel, then linked into
``paper_1702_00169_gb300/lib/libpdg.so``.  Host code is compiled with FP
contraction disabled so the plan coefficients are identical on x86-64 and
aarch64.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "lib")
OBJDIR = os.path.join(ROOT, "_build", "obj")
LIB = os.path.join(LIBDIR, "libpdg.so")

SOURCES = ["pdg_batch_df.cu", "pdg_batch.cu", "pdg_kernels_df.cu", "pdg_kernels.cu", "pdg_diag_df.cu",
           "pdg_diag.cu", "pdg_corner_df.cu", "pdg_corner.cu", "pdg_corner_tc.cu", "pdg_corner_hp.cu", "pdg_corner_hp_df.cu", "pdg_api.cu", "pdg_ctx.cu", "pdg_schedule.cu", "pdg_issue.cu", "pdg_autotune.cu",
           "pdg_batch_api.cu", "pdg_noalloc.cu", "pdg_probe.cu", "pdg_server.cu",
           "pdg_plan.cpp"]
# pass-kernel instantiations: one object per (number type, group of model variants)
INSTANCES = [("pdg_pass_inst.cu", f"pdg_pass_t{t}_g{g}", [f"-DPDG_INST_T={t}", f"-DPDG_INST_GROUP={g}"])
             for t in (1, 0) for g in (3, 2, 1, 0)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
          "-I", os.path.join(ROOT, "include")]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(job):
    src, name, defs = job if isinstance(job, tuple) else (job, os.path.splitext(job)[0], [])
    obj = os.path.join(OBJDIR, name + ".o")
    cmd = [nvcc()] + ARCH + COMMON + defs + ["-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd = [nvcc()] + COMMON + ["-x", "c++", "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(verbose=False):
    os.makedirs(OBJDIR, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    jobs = INSTANCES + SOURCES   # the slowest objects first
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(_compile, jobs))
    tmp = LIB + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
