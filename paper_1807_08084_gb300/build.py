"""In-tree build of the CUDA shared libraries with nvcc (sm_103a only).

    libzinv.so   csrc/*.cu  -- the C ABI of include/zinv.h
    libzsynth.so synth/synth.cu -- the GPU twin of the input generators
                 (compiled with -fmad=false so it matches the numpy twin bit for bit)

Translation units compile in parallel; a library is rebuilt when any of its
sources or headers is newer than it.  No --use_fast_math: division and square
root stay IEEE correctly rounded, as the paper's error analysis assumes (§3.3).
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
BUILD = PKG / "_build"
INCLUDE = ROOT / "include"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-cudart", "shared",
          f"-I{INCLUDE}", f"-I{PKG / 'csrc'}"]

LIBS = {
    "libzinv.so": {
        "sources": sorted((PKG / "csrc").glob("*.cu")),
        "deps": sorted((PKG / "csrc").glob("*.cuh")) + sorted(INCLUDE.glob("*.h")),
        "flags": [],
    },
    "libzsynth.so": {
        "sources": [PKG / "synth" / "synth.cu"],
        "deps": [],
        "flags": ["-fmad=false"],
    },
}


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not Path(exe).exists():
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libzinv")
    return exe


def _stale(out: Path, inputs) -> bool:
    if not out.exists():
        return True
    t = out.stat().st_mtime
    return any(Path(p).stat().st_mtime > t for p in inputs)


def build_lib(name: str, verbose: bool = False, ptxas_info: bool = False) -> Path:
    spec = LIBS[name]
    out = BUILD / name
    srcs = spec["sources"]
    if not _stale(out, list(srcs) + list(spec["deps"]) + [Path(__file__)]) and not ptxas_info:
        return out
    BUILD.mkdir(exist_ok=True)
    exe = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    objs = []

    def compile_one(src: Path):
        obj = BUILD / (src.stem + f".{os.getpid()}.o")
        cmd = [exe, *ARCH, *COMMON, *spec["flags"], *extra, "-c", str(src), "-o", str(obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src.name}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stdout + r.stderr

    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(compile_one, srcs))
    logs = []
    for obj, log in results:
        objs.append(obj)
        logs.append(log)
    tmp = BUILD / f"{name}.{os.getpid()}.tmp"
    cmd = [exe, *ARCH, "-shared", "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64",
           *map(str, objs), "-o", str(tmp)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link of {name} failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    for o in objs:
        o.unlink(missing_ok=True)
    if ptxas_info:
        (BUILD / f"{name}.ptxas.txt").write_text("\n".join(logs))
    if verbose:
        print(f"built {out}")
    return out


def build_all(verbose: bool = False, ptxas_info: bool = False) -> list[Path]:
    with ThreadPoolExecutor(max_workers=len(LIBS)) as ex:
        return list(ex.map(lambda n: build_lib(n, verbose, ptxas_info), LIBS))


if __name__ == "__main__":
    import sys
    for p in build_all(verbose=True, ptxas_info="-v" in sys.argv):
        print(p)
