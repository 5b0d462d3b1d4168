"""ctypes binding of libxflat (include/xflat.h).  Argument marshalling only: every step of the
radial integration runs in the library's CUDA kernels.  Importing this module loads the library
and raises if it is missing; there is no CPU fallback."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# XFLAT_VARIANT=bounds or sanitize loads that checking build (build.build(variant=...)) instead
_VARIANT = os.environ.get("XFLAT_VARIANT", "")
_LIB_PATH = os.path.join(_HERE, f"libxflat_{_VARIANT}.so" if _VARIANT else "libxflat.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is missing: run `python -c 'import __graft_entry__ as g; g.build()'`")
_lib = C.CDLL(_LIB_PATH)

ABI_VERSION = 2
OK, ERR_INVAL, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_NONFINITE, ERR_STEP, ERR_STATE, ERR_UNSUPPORTED = range(9)
FP64, MIXED = 0, 1
RK4, DP45, LIE_RK4, EXP_MIDPOINT, LIE_ADAPTIVE = 0, 1, 2, 3, 4
MATTER_NONE, MATTER_POWER_LAW, MATTER_CONSTANT, MATTER_TABLE = 0, 1, 2, 3
GEOMETRY_BULB, GEOMETRY_SINGLE_ANGLE, GEOMETRY_HOMOGENEOUS = 0, 1, 2
LAYOUT_MATRIX, LAYOUT_NATIVE = 0, 1

_INTEGRATORS = {"rk4": RK4, "dp45": DP45, "lie_rk4": LIE_RK4, "exp_midpoint": EXP_MIDPOINT,
                "lie_adaptive": LIE_ADAPTIVE}
_MATTER = {"none": MATTER_NONE, "power_law": MATTER_POWER_LAW, "constant": MATTER_CONSTANT,
           "table": MATTER_TABLE}
_GEOMETRY = {"bulb": GEOMETRY_BULB, "single_angle": GEOMETRY_SINGLE_ANGLE, "homogeneous": GEOMETRY_HOMOGENEOUS}
_PRECISION = {"fp64": FP64, "mixed": MIXED}


class xflat_config(C.Structure):
    _fields_ = [
        ("abi_version", C.c_uint32), ("n_flavor", C.c_uint32), ("n_energy", C.c_uint32),
        ("n_angle", C.c_uint32), ("precision", C.c_uint32), ("integrator", C.c_uint32),
        ("matter_kind", C.c_uint32), ("n_phi", C.c_uint32),
        ("R_km", C.c_double), ("E_min_MeV", C.c_double), ("E_max_MeV", C.c_double),
        ("dm2_eV2", C.c_double * 2), ("theta", C.c_double * 3),
        ("rtol", C.c_double), ("atol", C.c_double), ("h0_km", C.c_double),
        ("h_min_km", C.c_double), ("h_max_km", C.c_double), ("fixed_dr_km", C.c_double),
        ("rho0_gcc", C.c_double), ("r_ref_km", C.c_double), ("power", C.c_double), ("Ye", C.c_double),
        ("lambda_const_kmi", C.c_double),
        ("cuda_stream", C.c_void_p), ("barrier_timeout_ns", C.c_uint64),
        ("block_size", C.c_uint32), ("blocks_per_sm", C.c_uint32),
        ("steps_per_launch", C.c_uint32), ("geometry", C.c_uint32), ("mu_const_kmi", C.c_double),
    ]


class xflat_stats(C.Structure):
    _fields_ = [
        ("r_km", C.c_double), ("h_km", C.c_double), ("last_err", C.c_double),
        ("accepted", C.c_uint64), ("rejected", C.c_uint64), ("stage_evals", C.c_uint64),
        ("beam_stage_updates", C.c_uint64), ("launches", C.c_uint64),
        ("n_beams", C.c_uint32), ("n_instances", C.c_uint32), ("status", C.c_int32),
        ("grid_blocks", C.c_uint32), ("block_size", C.c_uint32),
    ]


_H = C.c_void_p
_P = C.c_void_p
_D = C.POINTER(C.c_double)
_SIGS = {
    "xflat_default_config": (C.POINTER(xflat_config),),
    "xflat_create": (C.POINTER(xflat_config), C.POINTER(_H)),
    "xflat_create_batch": (C.POINTER(xflat_config), C.c_uint32, C.POINTER(_H)),
    "xflat_destroy": (_H,),
    "xflat_set_spectra": (_H, _P, _P, _P),
    "xflat_set_spectra_inst": (_H, C.c_uint32, _P, _P, _P),
    "xflat_reset": (_H, C.c_double),
    "xflat_set_matter_table": (_H, C.c_uint32, _P, _P, C.c_uint32),
    "xflat_evolve": (_H, C.c_double, C.c_double),
    "xflat_evolve_batch": (_H, _P),
    "xflat_advance": (_H, _P, C.c_uint32, C.POINTER(C.c_int)),
    "xflat_advance_graph": (_H, C.c_uint32, C.c_uint32, C.POINTER(C.c_int)),
    "xflat_moments": (_H, _P, _P),
    "xflat_moments_inst": (_H, C.c_uint32, _P, _P),
    "xflat_moments_phi": (_H, C.c_uint32, _P, _P),
    "xflat_get_rho": (_H, _P, C.c_int, C.c_int),
    "xflat_get_rho_inst": (_H, C.c_uint32, _P, C.c_int, C.c_int),
    "xflat_set_rho": (_H, _P, C.c_int, C.c_int, C.c_double),
    "xflat_set_rho_inst": (_H, C.c_uint32, _P, C.c_int, C.c_int, C.c_double),
    "xflat_pee": (_H, _P, _P),
    "xflat_pee_inst": (_H, C.c_uint32, _P, _P),
    "xflat_flux_spectra": (_H, C.c_uint32, _P),
    "xflat_get_stats": (_H, C.POINTER(xflat_stats)),
    "xflat_get_stats_inst": (_H, C.c_uint32, C.POINTER(xflat_stats)),
    "xflat_adjoint": (_H, C.c_double, C.c_double, C.c_uint32, C.c_uint32, _P, _P, _P),
    "xflat_debug_barrier_extra": (_H, C.c_uint32),
    "xflat_debug_fail_alloc": (C.c_uint32,),
    "xflat_moments_2f_noalloc": (_P, C.c_uint32, C.c_uint32, _P, _P, _P, C.c_double, C.c_double,
                                 _P, _P),
    "xflat_debug_trace": (_H, C.c_uint32, _P, C.POINTER(C.c_uint32)),
    "xflat_create_shard": (C.POINTER(xflat_config), C.c_uint32, C.c_uint32, C.POINTER(_H)),
    "xflat_shard_info": (_H, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)),
    "xflat_shard_begin": (_H, C.c_double),
    "xflat_shard_pass": (_H, C.c_int32),
    "xflat_shard_partials": (_H, _P),
    "xflat_shard_set_totals": (_H, _P),
    "xflat_shard_serial": (_H, C.c_int32, C.POINTER(C.c_int)),
}
NOALLOC_MAX_ANGLES = 4096
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = list(_args)
    _f.restype = C.c_int
_lib.xflat_status_string.argtypes = [C.c_int]
_lib.xflat_status_string.restype = C.c_char_p
_lib.xflat_last_error.argtypes = [_H]
_lib.xflat_last_error.restype = C.c_char_p

# re-export the raw entry points under their C names
for _name in list(_SIGS) + ["xflat_status_string", "xflat_last_error"]:
    globals()[_name] = getattr(_lib, _name)


class XflatError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"xflat error {code} ({_lib.xflat_status_string(code).decode()}): {msg}")
        self.code = code


def _check(rc, h=None):
    if rc != OK:
        msg = _lib.xflat_last_error(h).decode() if h else ""
        raise XflatError(rc, msg)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def default_config() -> xflat_config:
    c = xflat_config()
    _check(_lib.xflat_default_config(C.byref(c)))
    return c


def config_from_workload(wl, **over) -> xflat_config:
    """Translate a bulb_inputs.Workload (or any object with the same attributes) into a config."""
    c = default_config()
    c.n_flavor, c.n_energy, c.n_angle = wl.n_flavor, wl.n_energy, wl.n_angle
    c.precision = _PRECISION[wl.precision]
    c.integrator = _INTEGRATORS[wl.integrator]
    c.matter_kind = _MATTER[wl.matter]
    c.R_km, c.E_min_MeV, c.E_max_MeV = wl.R_km, wl.E_min, wl.E_max
    c.dm2_eV2[0], c.dm2_eV2[1] = wl.dm2[0], wl.dm2[1]
    for i in range(3):
        c.theta[i] = wl.theta[i]
    c.rtol, c.atol, c.h0_km = wl.rtol, wl.atol, wl.h0
    if wl.n_steps:
        c.fixed_dr_km = (wl.r1 - wl.r0) / wl.n_steps
    c.rho0_gcc, c.r_ref_km, c.power, c.Ye = wl.rho0_gcc, wl.r_ref_km, wl.power, wl.Ye
    c.lambda_const_kmi = wl.lambda_const
    for k, v in over.items():
        if k == "precision" and isinstance(v, str):
            v = _PRECISION[v]
        if k == "integrator" and isinstance(v, str):
            v = _INTEGRATORS[v]
        if k == "geometry" and isinstance(v, str):
            v = _GEOMETRY[v]
        setattr(c, k, v)
    return c


class Solver:
    """Owning wrapper of one xflat handle (one instance or a batch; with `shard`, the beams
    [lo, hi) of one instance, advanced by the shard_* calls)."""

    def __init__(self, cfgs, stream=None, shard=None):
        if isinstance(cfgs, xflat_config):
            cfgs = [cfgs]
        arr = (xflat_config * len(cfgs))(*cfgs)
        if stream is not None:
            for c in arr:
                c.cuda_stream = stream
        self.h = _H()
        if shard is not None:
            if len(cfgs) != 1:
                raise ValueError("a beam shard belongs to one instance")
            _check(_lib.xflat_create_shard(arr, int(shard[0]), int(shard[1]), C.byref(self.h)))
        else:
            _check(_lib.xflat_create_batch(arr, len(cfgs), C.byref(self.h)))
        self.cfgs = list(arr)
        self.n_inst = len(cfgs)

    def close(self):
        if self.h:
            _lib.xflat_destroy(self.h)
            self.h = _H()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def nbeams(self, inst=0):
        c = self.cfgs[inst]
        return 2 * c.n_energy * c.n_angle * (c.n_phi if c.n_phi >= 2 else 1)

    def set_spectra(self, N, u=None, du=None, inst=0):
        N = np.ascontiguousarray(N, dtype=np.float64)
        u = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
        du = None if du is None else np.ascontiguousarray(du, dtype=np.float64)
        _check(_lib.xflat_set_spectra_inst(self.h, inst, _ptr(N), _ptr(u), _ptr(du)), self.h)

    def set_matter_table(self, r_km, lambda_kmi, inst=0):
        r = np.ascontiguousarray(r_km, dtype=np.float64)
        lam = np.ascontiguousarray(lambda_kmi, dtype=np.float64)
        _check(_lib.xflat_set_matter_table(self.h, inst, _ptr(r), _ptr(lam), len(r)), self.h)

    def reset(self, r0):
        _check(_lib.xflat_reset(self.h, r0), self.h)

    def evolve(self, r0, r1):
        _check(_lib.xflat_evolve(self.h, r0, r1), self.h)

    def evolve_batch(self, r1):
        r1 = np.ascontiguousarray(r1, dtype=np.float64)
        _check(_lib.xflat_evolve_batch(self.h, _ptr(r1)), self.h)

    def advance(self, r1=None, max_steps=1):
        done = C.c_int(0)
        r1p = None if r1 is None else np.ascontiguousarray(r1, dtype=np.float64)
        _check(_lib.xflat_advance(self.h, _ptr(r1p), max_steps, C.byref(done)), self.h)
        return bool(done.value)

    def advance_graph(self, n_launches, max_steps=1):
        done = C.c_int(0)
        _check(_lib.xflat_advance_graph(self.h, n_launches, max_steps, C.byref(done)), self.h)
        return bool(done.value)

    def moments(self, inst=0):
        n = self.cfgs[inst].n_flavor
        J0 = np.zeros(2 * n * n)
        J1 = np.zeros(2 * n * n)
        _check(_lib.xflat_moments_inst(self.h, inst, _ptr(J0), _ptr(J1)), self.h)
        return (J0[0::2] + 1j * J0[1::2]).reshape(n, n), (J1[0::2] + 1j * J1[1::2]).reshape(n, n)

    def moments_phi(self, inst=0):
        """Azimuthal moments (Jc, Js) of the extended bulb model, 2x2 complex."""
        Jc = np.zeros(8)
        Js = np.zeros(8)
        _check(_lib.xflat_moments_phi(self.h, inst, _ptr(Jc), _ptr(Js)), self.h)
        return (Jc[0::2] + 1j * Jc[1::2]).reshape(2, 2), (Js[0::2] + 1j * Js[1::2]).reshape(2, 2)

    def get_rho(self, layout=LAYOUT_MATRIX, inst=0, device_ptr=None):
        """Host copy (numpy) of the state, or a copy into device memory at device_ptr."""
        c = self.cfgs[inst]
        n, nb = c.n_flavor, self.nbeams(inst)
        if device_ptr is not None:
            _check(_lib.xflat_get_rho_inst(self.h, inst, C.c_void_p(device_ptr), 1, layout), self.h)
            return None
        if layout == LAYOUT_MATRIX:
            out = np.zeros(nb * 2 * n * n)
            _check(_lib.xflat_get_rho_inst(self.h, inst, _ptr(out), 0, layout), self.h)
            return (out[0::2] + 1j * out[1::2]).reshape(nb, n, n)
        nc = 3 if n == 2 else 9
        out = np.zeros((nc, nb))
        _check(_lib.xflat_get_rho_inst(self.h, inst, _ptr(out), 0, layout), self.h)
        return out

    def set_rho(self, rho, r, layout=LAYOUT_MATRIX, inst=0, device_ptr=None):
        if device_ptr is not None:
            _check(_lib.xflat_set_rho_inst(self.h, inst, C.c_void_p(device_ptr), 1, layout, r), self.h)
            return
        if layout == LAYOUT_MATRIX:
            rho = np.asarray(rho, dtype=np.complex128)
            flat = np.empty(rho.size * 2)
            flat[0::2] = rho.real.ravel()
            flat[1::2] = rho.imag.ravel()
        else:
            flat = np.ascontiguousarray(rho, dtype=np.float64)
        _check(_lib.xflat_set_rho_inst(self.h, inst, _ptr(flat), 0, layout, r), self.h)

    def pee(self, inst=0, per_beam=True):
        nb = self.nbeams(inst)
        out = np.zeros(nb) if per_beam else None
        mean = np.zeros(1)
        _check(_lib.xflat_pee_inst(self.h, inst, _ptr(out), _ptr(mean)), self.h)
        return out, float(mean[0])

    def flux_spectra(self, inst=0):
        """Number-flux energy spectra [2, n_flavor, n_energy] at the current radius."""
        c = self.cfgs[inst]
        out = np.zeros(2 * c.n_flavor * c.n_energy)
        _check(_lib.xflat_flux_spectra(self.h, inst, _ptr(out)), self.h)
        return out.reshape(2, c.n_flavor, c.n_energy)

    def stats(self, inst=0) -> xflat_stats:
        s = xflat_stats()
        _check(_lib.xflat_get_stats_inst(self.h, inst, C.byref(s)), self.h)
        return s

    def adjoint(self, r0, r1, n_steps, checkpoint_every=64):
        c = self.cfgs[0]
        dN = np.zeros(2 * c.n_flavor * c.n_energy)
        dth = np.zeros(1)
        J = np.zeros(1)
        _check(_lib.xflat_adjoint(self.h, r0, r1, n_steps, checkpoint_every, _ptr(dN), _ptr(dth),
                                  _ptr(J)), self.h)
        return float(J[0]), dN.reshape(2, c.n_flavor, c.n_energy), float(dth[0])

    # ---- beam shards (see shard.evolve_sharded) ----
    def shard_info(self):
        p, n = C.c_uint32(0), C.c_uint32(0)
        _check(_lib.xflat_shard_info(self.h, C.byref(p), C.byref(n)), self.h)
        return p.value, n.value

    def shard_begin(self, r1):
        _check(_lib.xflat_shard_begin(self.h, r1), self.h)

    def shard_pass(self, p):
        _check(_lib.xflat_shard_pass(self.h, p), self.h)

    def shard_partials(self):
        w = np.zeros(self.shard_info()[1], dtype=np.int64)
        _check(_lib.xflat_shard_partials(self.h, _ptr(w)), self.h)
        return w

    def shard_set_totals(self, w):
        w = np.ascontiguousarray(w, dtype=np.int64)
        _check(_lib.xflat_shard_set_totals(self.h, _ptr(w)), self.h)

    def shard_serial(self, after_moment_pass):
        done = C.c_int(0)
        _check(_lib.xflat_shard_serial(self.h, 1 if after_moment_pass else 0, C.byref(done)), self.h)
        return bool(done.value)

    def debug_barrier_extra(self, extra):
        _check(_lib.xflat_debug_barrier_extra(self.h, extra), self.h)
