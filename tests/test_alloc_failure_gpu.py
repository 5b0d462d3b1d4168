"""Allocation failures, injected on the host (xflat_debug_fail_alloc): every device or pinned-host
allocation that creating a handle makes is failed once in turn; each attempt must return
XFLAT_ERR_NOMEM or XFLAT_ERR_CUDA, leave the handle NULL and give back the device memory it had
taken.  A failure in a lazy allocation of an existing handle (the staging buffer of a state copy,
the matter table, the pass trace) fails that call only: the handle keeps working."""
import ctypes as C

import numpy as np
import pytest
import torch

from bulb_inputs import Workload
from oracle.physics import Grid

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _disarm(xf):
    yield
    xf.xflat_debug_fail_alloc(0)


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("precision,integrator", [("fp64", "dp45"), ("mixed", "dp45"), ("fp64", "rk4")])
def test_every_allocation_of_create_fails_cleanly(xf, precision, integrator):
    # 1M beams: the state planes and stage planes are tens of MB, so a leaked buffer shows
    wl = Workload(name="af", n_energy=500, n_angle=1000, integrator=integrator, precision=precision,
                  n_steps=10 if integrator == "rk4" else 0, r0=100.0, r1=101.0)
    cfg = xf.config_from_workload(wl)
    s = xf.Solver(cfg)                     # warm up the context and the library's kernels
    s.close()
    free0 = _free_bytes()
    n = 1
    while True:
        xf.xflat_debug_fail_alloc(n)
        h = C.c_void_p()
        rc = xf.xflat_create(C.byref(cfg), C.byref(h))
        xf.xflat_debug_fail_alloc(0)
        if rc == xf.OK:
            xf.xflat_destroy(h)
            break
        assert rc in (xf.ERR_NOMEM, xf.ERR_CUDA), (n, rc)
        assert not h.value, n
        n += 1
        assert n < 100
    assert n >= 12                        # the planes, the stage planes and every table failed once
    assert abs(_free_bytes() - free0) < 8 << 20


def test_lazy_allocation_failures_leave_the_handle_usable(xf):
    wl = Workload(name="af2", n_energy=37, n_angle=29, integrator="dp45", h0=0.5, matter="table",
                  matter_table_r=[11.0, 100.0, 1000.0], matter_table_lambda=[1e3, 10.0, 0.1])
    s = xf.Solver(xf.config_from_workload(wl))
    s.set_spectra(Grid.from_workload(wl).N)
    # the matter table's device copy
    xf.xflat_debug_fail_alloc(1)
    with pytest.raises(xf.XflatError) as e:
        s.set_matter_table(wl.matter_table_r, wl.matter_table_lambda)
    assert e.value.code in (xf.ERR_NOMEM, xf.ERR_CUDA)
    s.set_matter_table(wl.matter_table_r, wl.matter_table_lambda)
    s.reset(100.0)
    s.evolve(100.0, 101.0)
    ref = s.get_rho(xf.LAYOUT_NATIVE).copy()
    # the staging buffer of a state copy (first use on a fresh handle)
    t = xf.Solver(xf.config_from_workload(wl))
    t.set_spectra(Grid.from_workload(wl).N)
    t.set_matter_table(wl.matter_table_r, wl.matter_table_lambda)
    t.reset(100.0)
    t.evolve(100.0, 101.0)
    xf.xflat_debug_fail_alloc(1)
    with pytest.raises(xf.XflatError):
        t.get_rho(xf.LAYOUT_NATIVE)
    assert np.array_equal(t.get_rho(xf.LAYOUT_NATIVE), ref)
    # the pass trace
    xf.xflat_debug_fail_alloc(1)
    rc = xf.xflat_debug_trace(t.h, 4, None, None)
    assert rc in (xf.ERR_NOMEM, xf.ERR_CUDA)
    t.evolve(101.0, 102.0)
    s.evolve(101.0, 102.0)
    assert np.array_equal(t.get_rho(xf.LAYOUT_NATIVE), s.get_rho(xf.LAYOUT_NATIVE))
    s.close()
    t.close()
