"""Multi-rank logic on CPU ranks (torch.distributed, gloo, world size 2): sharding of beams and of
batch instances, the exact fixed-point moment exchange, and the slowest-rank timing reduction.

Each rank takes its shard of the same seeded state, forms its partial moments D = sum w t1 s and
J1 = sum w s in the device accumulators' fixed-point format, and the ranks exchange them; the
totals must be identical on every rank and bit-identical to the one-rank total, and agree with a
plain FP64 sum to the format's resolution.
"""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from bulb_inputs import Workload, batched_workloads, random_unit_states
from paper_1912_10596_gb300 import shard

R = 11.0


def contributions(seed=4, n_energy=37, n_angle=29, r=40.0):
    """Per-beam moment contributions (w t1 s, w s) of a random state, [n_beams, 6]."""
    wl = Workload(name="mr", n_energy=n_energy, n_angle=n_angle)
    N = wl.spectra()
    psi = random_unit_states(2, wl.n_beams, seed)
    s = np.stack([2 * (psi[:, 0] * np.conj(psi[:, 1])).real, -2 * (psi[:, 0] * np.conj(psi[:, 1])).imag,
                  np.abs(psi[:, 0]) ** 2 - np.abs(psi[:, 1]) ** 2], axis=1)
    u = (np.arange(n_angle) + 0.5) / n_angle
    du = np.full(n_angle, 1.0 / n_angle)
    ws = np.abs(N).sum()
    g = np.stack([(N[0, 0] - N[0, 1]) / ws, -(N[1, 0] - N[1, 1]) / ws])        # [2, n_energy]
    w = (du[None, :, None] * g[:, None, :]).reshape(-1)
    c = np.sqrt(1 - u * R * R / (r * r))
    t1 = np.broadcast_to(((1 - c) / c)[None, :, None], (2, n_angle, n_energy)).reshape(-1)
    return np.concatenate([(w * t1)[:, None] * s, w[:, None] * s], axis=1)


def fixed_partial(contrib, lo, hi):
    pairs = []
    for comp in range(contrib.shape[1]):
        acc = (0, 0)
        for x in contrib[lo:hi, comp]:
            acc = shard.fixed_add(acc, shard.to_fixed(float(x)))
        pairs.append(acc)
    return pairs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        contrib = contributions()
        lo, hi = shard.beam_shards(contrib.shape[0], world)[rank]
        total = shard.allreduce_fixed(fixed_partial(contrib, lo, hi))
        slowest = shard.max_over_ranks(1.5 + rank)
        out[rank] = (total, slowest)
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def two_rank_result():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
        return dict(out)


def test_exchange_is_exact_and_rank_independent(two_rank_result):
    contrib = contributions()
    one = fixed_partial(contrib, 0, contrib.shape[0])
    t0, t1 = two_rank_result[0][0], two_rank_result[1][0]
    assert t0 == t1 == one
    vals = np.array([shard.from_fixed(p) for p in t0])
    exact = np.array([math.fsum(contrib[:, c]) for c in range(contrib.shape[1])])
    # per beam the format truncates below 2^-64; the read-out hi + lo 2^-64 rounds once
    assert np.all(np.abs(vals - exact) <= contrib.shape[0] * 2.0**-64 + 2.0**-53 * np.abs(exact))


def test_slowest_rank_time(two_rank_result):
    assert two_rank_result[0][1] == two_rank_result[1][1] == 2.5


def test_beam_shards_cover_and_align():
    for n, world in ((4_000_000, 8), (2146, 2), (100, 4), (0, 3)):
        parts = shard.beam_shards(n, world)
        assert parts[0][0] == 0 and parts[-1][1] == n
        for (a, b), (c, d) in zip(parts, parts[1:]):
            assert b == c and a <= b
        assert all(lo % 128 == 0 for lo, _ in parts)


def test_instance_shards_balance():
    sizes = [wl.n_beams for wl in batched_workloads()]
    for world in (1, 2, 4, 8):
        parts = shard.instance_shards(sizes, world)
        assert sorted(i for p in parts for i in p) == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
        assert parts == shard.instance_shards(sizes, world)


def test_fixed_point_format():
    for x in (0.0, 1.0, -1.0, 0.3, -0.3, 1e-20, -1e-20, 12345.678, -2.0**-60):
        lo, hi = shard.to_fixed(x)
        assert 0 <= lo < 2**64
        assert hi * 2**64 + lo == int(x * 2.0**64)          # trunc(x 2^64), exactly
        assert abs(shard.from_fixed((lo, hi)) - x) <= 2.0**-64 + 2.0**-52 * max(1.0, abs(x))
    a, b = shard.to_fixed(0.75), shard.to_fixed(0.5)
    assert shard.from_fixed(shard.fixed_add(a, b)) == 1.25
    assert shard.from_fixed(shard.fixed_add(shard.to_fixed(-0.25), shard.to_fixed(0.25))) == 0.0


class FakeShard:
    """A stand-in for a beam-shard handle on a CPU rank: each 'pass' contributes this shard's part
    of fixed integer moments (and an error maximum), and the serial section finishes after a
    fixed number of steps; it records the totals it was handed."""

    def __init__(self, part, steps):
        self.part, self.steps, self.seen = part, steps, []
        self.step = 0

    def shard_info(self):
        return 3, 2 * self.part.shape[1] + 2

    def shard_begin(self, r1):
        self.step = 0

    def shard_pass(self, p):
        self.last = p

    def shard_partials(self):
        w = []
        for c in range(self.part.shape[1]):
            t = int(self.part[:, c].sum()) * (self.last + 2)
            w += [t % shard.TWO64 - (shard.TWO64 if t % shard.TWO64 >= 1 << 63 else 0), t >> 64]
        return w + [int(self.part.max()) * 0 + 7 + (self.last + 2), 0]

    def shard_set_totals(self, w):
        self.seen.append(list(w))

    def shard_serial(self, init):
        if not init:
            self.step += 1
        return self.step >= self.steps


def _sharded_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"], os.environ["MASTER_PORT"] = "127.0.0.1", str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(5)
        allp = rng.integers(-(1 << 60), 1 << 60, size=(64, 3))
        lo, hi = shard.beam_shards(64, world, align=4)[rank]
        fs = FakeShard(allp[lo:hi], steps=4)
        steps = shard.evolve_sharded([fs], 150.0, exchange=lambda w: shard.exchange_words(w))
        q.put((rank, steps, fs.seen))
    finally:
        dist.destroy_process_group()


def test_evolve_sharded_exchange_on_two_ranks():
    """The pass-by-pass driver on two gloo ranks: every rank is handed the same totals, equal to the
    one-rank totals of all beams (128-bit integer sums, error maximum by max), every pass."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_sharded_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict((r, (st, seen)) for r, st, seen in (q.get(timeout=120) for _ in ps))
    for p in ps:
        p.join(timeout=60)
    rng = np.random.default_rng(5)
    allp = rng.integers(-(1 << 60), 1 << 60, size=(64, 3))
    one = FakeShard(allp, steps=4)
    assert shard.evolve_sharded([one], 150.0) == 4
    assert res[0][0] == res[1][0] == 4
    assert res[0][1] == res[1][1] == one.seen
