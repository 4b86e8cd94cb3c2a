"""Build libpt.so, the sm_103a CUDA library behind include/pt.h, in-tree.

    python -m paper_2509_23043_gb300.build        (or build() from Python)

Each translation unit is compiled in parallel with nvcc for sm_103a only, then linked into a
shared library under paper_2509_23043_gb300/_build/.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
OUT_DIR = PKG / "_build"
LIB = OUT_DIR / "libpt.so"
# IsingFormer inference: its own library, as it links cuBLASLt for the plain projections
FORMER_LIB = OUT_DIR / "libptformer.so"
FORMER_SOURCES = ["pt_former.cu", "pt_gemm_tc.cu"]
CUDA_LIB_DIR = "/usr/local/cuda/lib64"
SOURCES = ["pt_api.cu", "pt_lattice.cu", "pt_lattice_gibbs.cu", "pt_lattice_big.cu", "pt_graph.cu", "pt_calib.cu"]
HEADERS = ["pt_device.cuh", "pt_layout.h", "pt_graph.cuh", "pt_lattice.cuh", "pt_gemm_tc.h", "pt_softmax2.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -ffp-contract=off on the host: FP64 threshold tables are evaluated exactly as written.
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
              "-Xptxas", "-O3"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpt.so")


def _stale() -> bool:
    if not LIB.exists() or not FORMER_LIB.exists():
        return True
    t = min(LIB.stat().st_mtime, FORMER_LIB.stat().st_mtime)
    deps = [CSRC / s for s in SOURCES + FORMER_SOURCES + HEADERS] + \
        [PKG.parent / "include" / "pt.h", PKG.parent / "include" / "pt_former.h"]
    return any(p.stat().st_mtime > t for p in deps)


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> Path:
    if not force and not _stale():
        return LIB
    OUT_DIR.mkdir(exist_ok=True)
    nvcc = _nvcc()
    flags = NVCC_FLAGS + list(extra_flags or [])

    def compile_one(src: str) -> Path:
        obj = OUT_DIR / (Path(src).stem + ".o")
        cmd = [nvcc, *ARCH, *flags, "-I", str(PKG.parent / "include"), "-c", str(CSRC / src),
               "-o", str(obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with ThreadPoolExecutor(len(SOURCES) + len(FORMER_SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES + FORMER_SOURCES))
    core, former = objs[:len(SOURCES)], objs[len(SOURCES):]
    for out, parts, libs in ((LIB, core, ["-lcudart"]),
                             (FORMER_LIB, former, ["-lcudart", f"-L{CUDA_LIB_DIR}", "-lcublasLt",
                                                   "-Xlinker", f"-rpath,{CUDA_LIB_DIR}"])):
        tmp = OUT_DIR / f"{out.stem}.{os.getpid()}.so"
        cmd = [nvcc, *ARCH, "-shared", "-o", str(tmp), *map(str, parts), *libs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed for {out.name}:\n{r.stderr}")
        os.replace(tmp, out)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
