"""Builds the CUDA library libbeor.so for sm_103a with nvcc (in-tree)."""

import concurrent.futures
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libbeor.so")
LIB_CHECKED = os.path.join(OUT_DIR, "libbeor_checked.so")
SOURCES = ["api.cu", "precompute.cu", "chol.cu", "mixed.cu", "mlp.cu", "noalloc.cu", "autotune.cu", "instrument.cu", "herk_tc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-warn-spills"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(verbose: bool = False, extra: list | None = None, variant: str = "regular") -> str:
    """Compile the library.  variant "regular": _build/libbeor.so;
    "checked": _build/libbeor_checked.so with the kernels' index checks
    (BEOR_BOUNDS_CHECK)."""
    nvcc = _nvcc()
    extra = list(extra or [])
    lib, obj_dir = LIB, OUT_DIR
    if variant == "checked":
        extra.append("-DBEOR_BOUNDS_CHECK")
        lib, obj_dir = LIB_CHECKED, os.path.join(OUT_DIR, "checked")
    elif variant != "regular":
        raise ValueError(variant)
    os.makedirs(obj_dir, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(obj_dir, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
