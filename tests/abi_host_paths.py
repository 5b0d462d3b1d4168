"""Drive every host-side argument path of the C ABI that needs no GPU: NULL handles and pointers
for every entry point, and seeded edge values and random mixtures of every configuration field
through xflat_create, xflat_create_batch and xflat_create_shard.  Run as a child process against
the sanitizer build (XFLAT_VARIANT=sanitize with the compiler's libasan preloaded), where any
out-of-bounds access, use after free or undefined behaviour in that code aborts the process.
Prints "host paths ok" and the number of calls on success."""
import ctypes as C
import math
import os
import random
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_1912_10596_gb300 import xflat as X  # noqa: E402

ALLOWED_CREATE = {X.ERR_INVAL, X.ERR_UNSUPPORTED, X.ERR_CUDA, X.ERR_NOMEM}
U32_EDGES = [0, 1, 2, 3, 4, 5, 7, 8, 63, 64, 65, 4096, 4097, 1 << 16, (1 << 31) - 1, 1 << 31, (1 << 32) - 1]
F64_EDGES = [0.0, -0.0, 1e-300, -1.0, 0.5, 1.0, 11.0, 1e300, -1e300, math.inf, -math.inf, math.nan]


def null_calls():
    n = 0
    for name, args in X._SIGS.items():
        vals = []
        for a in args:
            if a is C.c_double:
                vals.append(0.0)
            elif a in (C.c_uint32, C.c_int, C.c_int32, C.c_uint64):
                vals.append(0)
            else:
                vals.append(None)
        rc = getattr(X, name)(*vals)
        want = X.OK if name in ("xflat_destroy", "xflat_debug_fail_alloc") else X.ERR_INVAL
        assert rc == want, (name, rc)
        n += 1
    for code in range(-3, 20):
        assert X.xflat_status_string(code)
        n += 1
    assert X.xflat_last_error(None) is not None
    return n + 1


def create(cfg):
    h = C.c_void_p()
    rc = X.xflat_create(C.byref(cfg), C.byref(h))
    if rc == X.OK:                  # only on a machine with a GPU
        X.xflat_destroy(h)
    else:
        assert rc in ALLOWED_CREATE, rc
        assert not h.value, "a failed create must leave the handle NULL"
    return rc


def field_edges():
    n = 0
    for fname, ftype in X.xflat_config._fields_:
        if fname in ("abi_version", "cuda_stream"):
            continue
        if ftype is C.c_double:
            values = F64_EDGES
        elif isinstance(ftype, type) and issubclass(ftype, C.Array):
            values = F64_EDGES
        elif ftype is C.c_uint64:
            values = [0, 1, (1 << 64) - 1]
        else:
            values = U32_EDGES
        for v in values:
            cfg = X.default_config()
            if isinstance(getattr(cfg, fname), C.Array):
                arr = getattr(cfg, fname)
                for i in range(len(arr)):
                    arr[i] = v
            else:
                setattr(cfg, fname, v)
            create(cfg)
            n += 1
    return n


def random_mixtures(count, seed):
    rng = random.Random(seed)
    n = 0
    for _ in range(count):
        cfg = X.default_config()
        for fname, ftype in X.xflat_config._fields_:
            if fname in ("abi_version", "cuda_stream") or rng.random() < 0.7:
                continue
            if ftype is C.c_double:
                setattr(cfg, fname, rng.choice(F64_EDGES + [rng.uniform(-1e3, 1e3)]))
            elif isinstance(ftype, type) and issubclass(ftype, C.Array):
                arr = getattr(cfg, fname)
                for i in range(len(arr)):
                    arr[i] = rng.choice(F64_EDGES)
            elif ftype is C.c_uint64:
                setattr(cfg, fname, rng.choice([0, 1, (1 << 64) - 1, rng.getrandbits(64)]))
            else:
                setattr(cfg, fname, rng.choice(U32_EDGES + [rng.getrandbits(32), rng.randrange(0, 9)]))
        create(cfg)
        n += 1
    return n


def batch_and_shard():
    n = 0
    h = C.c_void_p()
    cfgs = (X.xflat_config * 3)()
    for i in range(3):
        C.memmove(C.byref(cfgs[i]), C.byref(X.default_config()), C.sizeof(X.xflat_config))
    cfgs[1].n_flavor = 3                       # mixed flavour counts in one batch
    rc = X.xflat_create_batch(cfgs, 3, C.byref(h))
    assert rc in ALLOWED_CREATE and not h.value, rc
    cfgs[1].n_flavor = 2
    cfgs[2].precision = X.MIXED                # mixed precisions in one batch
    rc = X.xflat_create_batch(cfgs, 3, C.byref(h))
    assert rc in ALLOWED_CREATE and not h.value, rc
    assert X.xflat_create_batch(cfgs, 0, C.byref(h)) == X.ERR_INVAL
    n += 3
    cfg = X.default_config()
    nb = 2 * cfg.n_energy * cfg.n_angle
    for lo, hi in [(0, 0), (3, 64), (64, 3), (0, nb + 4), (nb, nb), ((1 << 32) - 4, (1 << 32) - 1),
                   (4, 6), (0, nb)]:
        rc = X.xflat_create_shard(C.byref(cfg), lo, hi, C.byref(h))
        if rc == X.OK:
            X.xflat_destroy(h)
        else:
            assert rc in ALLOWED_CREATE and not h.value, (lo, hi, rc)
        n += 1
    return n


def noalloc_paths():
    buf = (C.c_double * 64)()
    p = C.cast(buf, C.c_void_p)
    n = 0
    for nb, na in [(0, 0), (1, 1), (16, X.NOALLOC_MAX_ANGLES + 1), ((1 << 32) - 1, 1)]:
        rc = X.xflat_moments_2f_noalloc(None, nb, na, p, p, p, 11.0, 11.0, p, None)
        assert rc == X.ERR_INVAL, rc
        n += 1
    for r in (math.nan, -1.0, 0.0, 5.0):
        rc = X.xflat_moments_2f_noalloc(p, 4, 1, p, p, p, 11.0, r, p, None)   # r < R or NaN: no launch
        assert rc == X.ERR_INVAL, rc
        n += 1
    return n


def main():
    assert os.path.basename(X._LIB_PATH) == "libxflat_sanitize.so", X._LIB_PATH
    with open("/proc/self/maps") as f:
        assert "libasan" in f.read(), "AddressSanitizer runtime not loaded"
    n = null_calls() + field_edges() + random_mixtures(400, 20191223) + batch_and_shard() + noalloc_paths()
    print(f"host paths ok {n}")


if __name__ == "__main__":
    main()
