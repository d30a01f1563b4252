"""In-tree build of the native libraries.

* ``libftle.so``        - the CUDA kernels and the C-ABI (``include/ftle.h``), built by nvcc
                          for sm_103a only.
* ``libftle_inputs.so`` - the seeded mesh/neighbour generator (plain C, host only).

Each library is rebuilt when any of its sources is newer than the shared object.
Builds are serialised with a file lock, so parallel test workers do not race.
"""
from __future__ import annotations

import fcntl
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INPUTS = PKG / "inputs"
INCLUDE = ROOT / "include"

LIBFTLE = CSRC / "libftle.so"
LIBINPUTS = INPUTS / "libftle_inputs.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xptxas", "-warn-spills"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libftle.so")


def _stale(target: Path, sources: list[Path]) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(s.stat().st_mtime > t for s in sources)


def _run(cmd: list[str], cwd: Path) -> None:
    proc = subprocess.run(cmd, cwd=cwd, capture_output=True, text=True)
    if proc.returncode != 0:
        raise RuntimeError(f"build step failed: {' '.join(cmd)}\n{proc.stdout}\n{proc.stderr}")


class _Lock:
    def __init__(self, path: Path):
        self.path = path

    def __enter__(self):
        self.fd = open(self.path, "w")
        fcntl.flock(self.fd, fcntl.LOCK_EX)
        return self

    def __exit__(self, *exc):
        fcntl.flock(self.fd, fcntl.LOCK_UN)
        self.fd.close()


def build_inputs(force: bool = False) -> Path:
    src = [INPUTS / "meshgen.c"]
    with _Lock(INPUTS / ".build.lock"):
        if force or _stale(LIBINPUTS, src):
            tmp = LIBINPUTS.with_suffix(".so.tmp")
            _run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-ffp-contract=off", "-o", str(tmp),
                  *map(str, src)], INPUTS)
            os.replace(tmp, LIBINPUTS)
    return LIBINPUTS


def cuda_sources() -> list[Path]:
    return sorted(CSRC.glob("*.cu"))


def cuda_headers() -> list[Path]:
    return sorted(CSRC.glob("*.cuh")) + sorted(INCLUDE.glob("*.h"))


def build_ftle(force: bool = False, jobs: int | None = None) -> Path:
    """Compile every ``csrc/*.cu`` for sm_103a (in parallel) and link ``libftle.so``."""
    srcs = cuda_sources()
    deps = srcs + cuda_headers()
    with _Lock(CSRC / ".build.lock"):
        if not (force or _stale(LIBFTLE, deps)):
            return LIBFTLE
        nvcc = _nvcc()
        objdir = CSRC / "_build"
        objdir.mkdir(exist_ok=True)
        inc = ["-I", str(INCLUDE), "-I", str(CSRC)]

        def compile_one(s: Path) -> Path:
            obj = objdir / (s.stem + ".o")
            _run([nvcc, *ARCH, *NVCC_FLAGS, *inc, "-c", str(s), "-o", str(obj)], CSRC)
            return obj

        with ThreadPoolExecutor(max_workers=jobs or min(8, max(1, len(srcs)))) as ex:
            objs = list(ex.map(compile_one, srcs))
        tmp = LIBFTLE.with_suffix(".so.tmp")
        _run([nvcc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs), "-lcudart"], CSRC)
        os.replace(tmp, LIBFTLE)
    return LIBFTLE


def build_all(force: bool = False) -> None:
    build_inputs(force)
    build_ftle(force)
