"""Build libpty.so in-tree with nvcc for sm_103a (GB300).

Each translation unit under csrc/ compiles in parallel to an object file, then nvcc links
the shared library.  The output is cached under _lib/ by a hash of the sources and flags.
"""
from __future__ import annotations

import glob
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIBDIR = os.path.join(HERE, "_lib")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC]
# extra nvcc flags (space-separated), e.g. compile-time tuning defines; part of the cache key
FLAGS += os.environ.get("PTY_NVCC_FLAGS", "").split()


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpty")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _digest(extra=()):
    h = hashlib.sha1()
    for f in sorted(glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INCLUDE, "*.h"))):
        h.update(os.path.basename(f).encode())
        h.update(open(f, "rb").read())
    h.update(" ".join(ARCH + FLAGS + list(extra)).encode())
    return h.hexdigest()[:16]


def lib_path() -> str:
    return os.path.join(LIBDIR, f"libpty-{_digest()}.so")


def _prune(keep: str) -> None:
    """Delete every superseded build product under _lib/ (older libraries, partial links,
    object folders of earlier or failed builds), keeping only ``keep``."""
    if not os.path.isdir(LIBDIR):
        return
    for name in os.listdir(LIBDIR):
        path = os.path.join(LIBDIR, name)
        if path == keep:
            continue
        if name.startswith("obj-") and os.path.isdir(path):
            # another process may be compiling into its own obj-<pid> right now
            pid = name[4:]
            if pid.isdigit() and int(pid) != os.getpid() and _alive(int(pid)):
                continue
            shutil.rmtree(path, ignore_errors=True)
        elif name.startswith("libpty-") and (name.endswith(".so") or ".so.tmp" in name):
            if ".so.tmp" in name:
                pid = name.rsplit(".so.tmp", 1)[1]
                if pid.isdigit() and int(pid) != os.getpid() and _alive(int(pid)):
                    continue
            try:
                os.remove(path)
            except OSError:
                pass


def _alive(pid: int) -> bool:
    try:
        os.kill(pid, 0)
    except ProcessLookupError:
        return False
    except PermissionError:
        return True
    return True


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    """Compile (if needed) and return the path of libpty.so.

    Only the current library is kept under _lib/: every earlier build (a different source
    hash) and every object folder is deleted after a successful link, and the object
    folder of this build is deleted whether or not nvcc succeeds.
    """
    out = lib_path()
    if os.path.exists(out) and not force:
        _prune(out)
        return out
    os.makedirs(LIBDIR, exist_ok=True)
    tmpdir = os.path.join(LIBDIR, f"obj-{os.getpid()}")
    os.makedirs(tmpdir, exist_ok=True)
    try:
        cc = nvcc()
        extra = ["-Xptxas", "-v"] if ptxas_verbose else []
        procs, objs = [], []
        for src in _sources():
            obj = os.path.join(tmpdir, os.path.basename(src) + ".o")
            cmd = [cc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
            objs.append(obj)
        failed = []
        for src, p in procs:
            o, _ = p.communicate()
            if p.returncode != 0 or (ptxas_verbose and o):
                sys.stderr.write(o.decode(errors="replace"))
            if p.returncode != 0:
                failed.append(src)
        if failed:
            raise RuntimeError(f"nvcc failed for {failed}")
        tmp = out + f".tmp{os.getpid()}"
        cmd = [cc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-lcudart_static", "-lrt",
               "-ldl", "-lpthread"]
        try:
            subprocess.run(cmd, check=True)
            os.replace(tmp, out)
        finally:
            if os.path.exists(tmp):
                os.remove(tmp)
    finally:
        shutil.rmtree(tmpdir, ignore_errors=True)
    _prune(out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_verbose="-v" in sys.argv))
