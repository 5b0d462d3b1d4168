"""Launch shapes of the persistent step kernel: every resident-block count the mixed two-flavour
kernels are built for is reached on the GPU, with the shared memory the tables and the state ring
take (a kernel that no longer fits would silently run with fewer blocks per SM), and the defaults
follow the state size: one 512-thread block per SM while both state buffers fit the L2, two
256-thread blocks per SM once they do not."""
import pytest
import torch

from bulb_inputs import Workload, batched_workloads, workload_2f_large
from oracle.physics import Grid

pytestmark = pytest.mark.gpu


def _solver(xf, wls, **over):
    s = xf.Solver([xf.config_from_workload(w, **over) for w in wls])
    for i, w in enumerate(wls):
        s.set_spectra(Grid.from_workload(w).N, inst=i)
    return s


def _sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("block,bps", [(512, 1), (256, 2), (256, 3)])
def test_mixed_kernels_reach_their_resident_blocks(xf, block, bps):
    wl = workload_2f_large("mixed")
    s = _solver(xf, [wl], block_size=block, blocks_per_sm=bps)
    st = s.stats()
    assert (st.block_size, st.grid_blocks) == (block, bps * _sms())
    s.close()


def test_extended_kernel_reaches_two_blocks_per_sm(xf):
    wl = Workload(name="ext", n_energy=100, n_angle=2000, integrator="dp45", precision="mixed", rtol=1e-6,
                  atol=1e-6)
    s = _solver(xf, [wl], n_phi=10)
    st = s.stats()
    assert (st.block_size, st.grid_blocks) == (256, 2 * _sms())
    s.close()


def test_default_shapes_follow_the_state_size(xf):
    s = _solver(xf, [workload_2f_large("mixed")])          # 96 MB of state: fits the L2
    st = s.stats()
    assert (st.block_size, st.grid_blocks) == (512, _sms())
    s.close()
    s = _solver(xf, batched_workloads())                   # 676 MB of state: streams from HBM
    st = s.stats()
    assert (st.block_size, st.grid_blocks) == (256, 2 * _sms())
    s.close()
