"""Small runs of every step-kernel family through the library the binding loads (XFLAT_VARIANT
selects a checking build): two and three flavours (three also with the adaptive exponential
integrator), FP64 and mixed precision, each integrator, the
extended bulb model, the single-angle geometry with a matter table, a batch of uneven instances
(dynamic piece scheduling) and two beam shards, each over a ragged beam count.  `run_cases()`
returns the final states and moments by case name; as a script it writes them to an .npz file, so
that a checking build running in a child process can be compared with the plain build."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

from bulb_inputs import Workload  # noqa: E402
from oracle.physics import Grid  # noqa: E402  (input binning only: the spectra table)


def _solver(xf, wl, **over):
    s = xf.Solver(xf.config_from_workload(wl, **over))
    s.set_spectra(Grid.from_workload(wl).N)
    if wl.matter == "table":
        s.set_matter_table(wl.matter_table_r, wl.matter_table_lambda)
    return s


def _single(xf, out, name, wl, r0, r1, **over):
    s = _solver(xf, wl, **over)
    s.reset(r0)
    s.evolve(r0, r1)
    out[name + "/rho"] = s.get_rho(xf.LAYOUT_NATIVE)
    out[name + "/mom"] = np.concatenate([np.ravel(m) for m in s.moments()])
    st = s.stats()
    out[name + "/steps"] = np.array([st.accepted, st.rejected])
    s.close()


def run_cases(xf):
    out = {}
    ragged = dict(n_energy=37, n_angle=29)
    # windows at 100 km, where the explicit steps of the adaptive schemes are not yet tiny
    _single(xf, out, "fp64_rk4", Workload(name="c1", n_steps=12, r0=100.0, r1=101.134, **ragged), 100.0, 101.134)
    _single(xf, out, "fp64_dp45", Workload(name="c2", integrator="dp45", h0=0.05, **ragged), 100.0, 101.0)
    _single(xf, out, "mixed_dp45", Workload(name="c3", integrator="dp45", precision="mixed", rtol=1e-6,
                                            atol=1e-6, h0=0.05, **ragged), 100.0, 101.0)
    _single(xf, out, "mixed_lie", Workload(name="c4", integrator="lie_adaptive", precision="mixed", rtol=1e-6,
                                           atol=1e-6, h0=0.05, **ragged), 100.0, 101.0)
    _single(xf, out, "fp64_lie_rk4", Workload(name="c5", integrator="lie_rk4", n_steps=10, r0=100.0, r1=101.0,
                                              **ragged), 100.0, 101.0)
    _single(xf, out, "fp64_em2", Workload(name="c6", integrator="exp_midpoint", h0=0.05, **ragged), 100.0, 101.0)
    _single(xf, out, "fp64_3f", Workload(name="c7", n_flavor=3, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.78),
                                         integrator="dp45", h0=0.05, n_energy=13, n_angle=11), 100.0, 100.5)
    _single(xf, out, "mixed_ext", Workload(name="c8", integrator="dp45", precision="mixed", rtol=1e-6, atol=1e-6,
                                           h0=0.05, n_energy=13, n_angle=11), 100.0, 100.5, n_phi=4)
    _single(xf, out, "fp64_3f_lie", Workload(name="c10", n_flavor=3, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.78),
                                             integrator="lie_adaptive", h0=0.05, n_energy=13, n_angle=11),
            100.0, 100.5)
    _single(xf, out, "mixed_3f_lie", Workload(name="c11", n_flavor=3, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.78),
                                              integrator="lie_adaptive", precision="mixed", rtol=1e-6, atol=1e-6,
                                              h0=0.05, n_energy=13, n_angle=11), 100.0, 100.5)
    rt = [11.0, 50.0, 200.0, 1000.0]
    _single(xf, out, "fp64_single_table",
            Workload(name="c9", integrator="dp45", h0=0.05, matter="table", matter_table_r=rt,
                     matter_table_lambda=[1e3, 40.0, 2.0, 0.01], **ragged), 100.0, 102.0, geometry="single_angle")
    # a batch of uneven instances (dynamic piece scheduling)
    wls = [Workload(name="b0", integrator="dp45", h0=0.5, **ragged),
           Workload(name="b1", integrator="dp45", h0=0.5, n_energy=11, n_angle=7, matter="power_law"),
           Workload(name="b2", integrator="dp45", h0=0.2, n_energy=64, n_angle=3)]
    s = xf.Solver([xf.config_from_workload(w) for w in wls])
    for i, w in enumerate(wls):
        s.set_spectra(Grid.from_workload(w).N, inst=i)
    s.reset(100.0)
    s.evolve_batch([104.0, 104.0, 104.0])
    for i in range(len(wls)):
        out[f"batch{i}/rho"] = s.get_rho(xf.LAYOUT_NATIVE, inst=i)
    s.close()
    # two beam shards of one problem
    from paper_1912_10596_gb300 import shard
    wl = Workload(name="sh", integrator="dp45", h0=0.5, **ragged)
    n = wl.n_beams
    parts = []
    for lo, hi in [(0, 1024), (1024, n)]:
        p = xf.Solver(xf.config_from_workload(wl), shard=(lo, hi))
        p.set_spectra(Grid.from_workload(wl).N)
        p.reset(100.0)
        parts.append(p)
    shard.evolve_sharded(parts, 102.0)
    out["shard/rho"] = np.concatenate([parts[0].get_rho(xf.LAYOUT_NATIVE)[:, :1024],
                                       parts[1].get_rho(xf.LAYOUT_NATIVE)[:, 1024:]], axis=1)
    for p in parts:
        p.close()
    return out


if __name__ == "__main__":
    from paper_1912_10596_gb300 import xflat
    res = run_cases(xflat)
    np.savez(sys.argv[1], **res)
    print(f"cases ok {len(res)} {os.path.basename(xflat._LIB_PATH)}")
