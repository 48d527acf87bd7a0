"""Build libcbp.so (the CUDA library behind include/cbp.h) in-tree for sm_103a.

Each .cu file under csrc/ compiles to an object in parallel; the objects link
into ``paper_1203_4874_gb300/libcbp.so``.  The same sources compiled with
-DCBP_CHECKS link into ``libcbp_checks.so``, the bounds-checked diagnostic
build (cbp_check_words); both builds' objects compile in one parallel pool.
Rebuilds only when a source or header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
BUILD = PKG / "_build"
LIB = PKG / "libcbp.so"
# variant -> (object folder, library, extra flags)
VARIANTS = {"release": (BUILD, LIB, []),
            "checks": (PKG / "_build_checks", PKG / "libcbp_checks.so", ["-DCBP_CHECKS"])}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-O3"]


def _nvcc() -> str:
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = Path(cuda) / "bin" / "nvcc"
    return str(p) if p.exists() else "nvcc"


def _sources():
    return sorted(CSRC.glob("*.cu"))


def _stale(lib: Path = LIB) -> bool:
    if not lib.exists():
        return True
    t = lib.stat().st_mtime
    deps = list(CSRC.glob("*")) + list(INCLUDE.glob("*.h")) + [Path(__file__)]
    return any(d.stat().st_mtime > t for d in deps)


def _extra_flags() -> list:
    """Extra nvcc flags from CBP_NVCC_FLAGS (e.g. -DCBP_PHASE_TIMING for a
    build that prints per-phase cycle counts of the solver kernels)."""
    return os.environ.get("CBP_NVCC_FLAGS", "").split()


def _compile(src: Path, verbose_ptxas: bool, variant: str = "release") -> Path:
    folder, _, flags = VARIANTS[variant]
    obj = folder / (src.stem + ".o")
    cmd = [_nvcc(), *ARCH, *NVCC_FLAGS, *flags, *_extra_flags(), f"-I{INCLUDE}", f"-I{CSRC}", "-c",
           str(src), "-o", str(obj)]
    if verbose_ptxas:
        cmd[1:1] = ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src.name}:\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas:
        sys.stderr.write(r.stderr)
    return obj


def _link(objs, lib: Path) -> None:
    tmp = lib.with_suffix(".so.tmp")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cmd = [_nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", str(tmp), *map(str, objs),
           "-Xlinker", f"-rpath={cuda}/lib64", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)


def build(force: bool = False, verbose_ptxas: bool = False, variants=("release", "checks")) -> Path:
    """Compile and link the libraries of `variants` that are out of date
    (all of them with force); returns the release library's path."""
    todo = [v for v in variants if force or _stale(VARIANTS[v][1])]
    if not todo:
        return LIB
    srcs = _sources()
    jobs = [(v, src) for v in todo for src in srcs]
    for v in todo:
        VARIANTS[v][0].mkdir(exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(lambda j: (j[0], _compile(j[1], verbose_ptxas, j[0])), jobs))
    for v in todo:
        _link([o for vv, o in objs if vv == v], VARIANTS[v][1])
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv)
    print(LIB)
