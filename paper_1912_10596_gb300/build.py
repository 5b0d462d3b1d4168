"""Build the in-tree CUDA library libxflat.so for sm_103a with nvcc (no cmake, parallel TUs).

Two checking variants build beside it from the same sources (``build(variant=...)``), each into its
own library that the binding loads when XFLAT_VARIANT names it:

* ``bounds`` (libxflat_bounds.so): -DXFLAT_BOUNDS, the step kernel tests every plane, stage-plane,
  table and piece access of its pass body against the allocation it has to fall in, skips an access
  outside and reports the first as XFLAT_ERR_CUDA with its site;
* ``sanitize`` (libxflat_sanitize.so): the host code of the C ABI (api.cu, noalloc.cu) under
  AddressSanitizer and UndefinedBehaviorSanitizer (any finding aborts), linked with the plain
  build's kernel objects; load it with the compiler's libasan preloaded.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libxflat.so")
STAMP = LIB + ".sha256"      # fingerprint of the inputs the present libxflat.so was built from
SOURCES = ["api.cu", "kernels_2f.cu", "kernels_lie.cu", "kernels_2e.cu", "kernels_3f.cu", "kernels_3f_lie.cu",
           "adjoint_2f.cu", "noalloc.cu"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC", "-diag-suppress", "128",
              "-Xptxas", "-v"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


# variant: (extra compile flags, extra link flags, the sources compiled with them or None for all;
# the others are the plain build's objects).  nvcc splits an -Xcompiler value at commas, so each
# sanitizer goes in its own flag.
_SAN = ["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined", "-Xcompiler",
        "-fsanitize=float-cast-overflow"]
VARIANTS = {
    "bounds": (["-DXFLAT_BOUNDS"], [], None),
    "sanitize": (_SAN + ["-Xcompiler", "-fno-sanitize-recover=all", "-Xcompiler", "-fno-omit-frame-pointer",
                         "-Xcompiler", "-g"], _SAN, ["api.cu", "noalloc.cu"]),
}


def lib_path(variant: str | None = None) -> str:
    """The library file of the plain build (None) or of a checking variant."""
    if variant is None:
        return LIB
    if variant not in VARIANTS:
        raise ValueError(f"unknown build variant {variant!r} (known: {sorted(VARIANTS)})")
    return os.path.join(HERE, f"libxflat_{variant}.so")


def _compile(src: str, build_dir: str = BUILD, extra: tuple = ()) -> tuple[str, str]:
    obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc(), *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    with open(os.path.join(build_dir, src + ".ptxas.txt"), "w") as f:
        f.write(res.stderr)
    return obj, res.stderr


def sources() -> list[str]:
    return [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _fingerprint(extra: tuple = ()) -> str:
    """SHA-256 over every file of csrc/, the public header, this script and the nvcc flags: the
    library is rebuilt whenever any of them differs from what the present binary was built from
    (file times are not trusted: a copied tree can carry a binary newer than its sources)."""
    h = hashlib.sha256()
    deps = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC))
    deps += [os.path.join(HERE, "..", "include", "xflat.h"), os.path.abspath(__file__)]
    for d in deps:
        if os.path.isfile(d):
            h.update(os.path.basename(d).encode() + b"\0")
            with open(d, "rb") as f:
                h.update(f.read())
    h.update("\0".join(NVCC_FLAGS + list(extra) + SOURCES).encode())
    return h.hexdigest()


def _stale(fp: str, lib: str = LIB) -> bool:
    stamp = lib + ".sha256"
    if not os.path.exists(lib) or not os.path.exists(stamp):
        return True
    with open(stamp) as f:
        return f.read().strip() != fp


def build(force: bool = False, verbose: bool = False, variant: str | None = None) -> str:
    """Compile every CUDA translation unit for sm_103a and link libxflat.so in the package (or,
    with `variant`, the checking library of that name)."""
    lib = lib_path(variant)
    cflags, lflags, only = VARIANTS[variant] if variant else ([], [], None)
    build_dir = BUILD if variant is None else os.path.join(BUILD, variant)
    fp = _fingerprint(tuple(cflags + lflags + (only or [])))
    if not force and not _stale(fp, lib):
        return lib
    if only is not None:
        build(verbose=verbose)            # the plain objects this variant links
    os.makedirs(build_dir, exist_ok=True)
    srcs = sources()
    mine = [s for s in srcs if only is None or s in only]
    with cf.ThreadPoolExecutor(max_workers=min(len(mine), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(s, build_dir, tuple(cflags)), mine))
    built = {s: o for s, (o, _) in zip(mine, results)}
    objs = [built.get(s, os.path.join(BUILD, os.path.splitext(s)[0] + ".o")) for s in srcs]
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    tmp = lib + ".tmp"
    cmd = [_nvcc(), "-shared", "-gencode", "arch=compute_103a,code=sm_103a", *lflags, "-o", tmp, *objs,
           "-lcudart"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib)
    with open(lib + ".sha256", "w") as f:
        f.write(fp + "\n")
    return lib


if __name__ == "__main__":
    var = next((a.split("=", 1)[1] for a in sys.argv if a.startswith("--variant=")), None)
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, variant=var))
