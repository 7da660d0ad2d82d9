"""In-tree build of the package's native libraries.

* ``libdawn.so``          -- the CUDA path (``csrc/*.cu``) behind the C ABI of
  ``include/dawn.h``, compiled for sm_103a only.
* ``libdawn_graphgen.so`` -- the seeded synthetic graph generators (plain C).

Both land in ``paper_2208_04514_b300/_lib``.  A library is rebuilt when any of
its sources or headers is newer than the built file.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
LIB_DIR = PKG / "_lib"
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"

DAWN_SO = LIB_DIR / "libdawn.so"
GRAPHGEN_SO = LIB_DIR / "libdawn_graphgen.so"

NVCC_ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the CUDA path cannot be built")


def _stale(target: Path, deps: list[Path]) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(d.stat().st_mtime > t for d in deps)


def _run(cmd: list[str]) -> None:
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"build failed: {' '.join(cmd)}\n{res.stdout}\n{res.stderr}")


def dawn_sources() -> list[Path]:
    return sorted(CSRC.glob("*.cu"))


def build_dawn(force: bool = False, extra_flags: list[str] | None = None,
               out: Path | None = None) -> Path:
    """Compile ``csrc/*.cu`` into one shared library for sm_103a."""
    out = out or DAWN_SO
    srcs = dawn_sources()
    deps = srcs + sorted(CSRC.glob("*.cuh")) + sorted(INCLUDE.glob("*.h")) + [Path(__file__)]
    if not force and not extra_flags and not _stale(out, deps):
        return out
    LIB_DIR.mkdir(parents=True, exist_ok=True)
    tmp = out.with_suffix(".so.tmp")
    cmd = [_nvcc(), *NVCC_ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared",
           "-Xcompiler", "-fPIC,-fvisibility=hidden", "-I", str(INCLUDE),
           "-o", str(tmp), *map(str, srcs), *(extra_flags or [])]
    _run(cmd)
    tmp.replace(out)
    return out


def build_graphgen(force: bool = False) -> Path:
    src = PKG / "graphgen" / "graphgen.c"
    if not force and not _stale(GRAPHGEN_SO, [src, Path(__file__)]):
        return GRAPHGEN_SO
    LIB_DIR.mkdir(parents=True, exist_ok=True)
    tmp = GRAPHGEN_SO.with_suffix(".so.tmp")
    _run(["gcc", "-O2", "-std=c11", "-fPIC", "-fopenmp", "-shared", "-o", str(tmp), str(src), "-lm"])
    tmp.replace(GRAPHGEN_SO)
    return GRAPHGEN_SO


def build_all(force: bool = False) -> None:
    build_graphgen(force)
    build_dawn(force)


if __name__ == "__main__":
    import sys
    build_all(force="--force" in sys.argv)
    print(DAWN_SO, GRAPHGEN_SO)
