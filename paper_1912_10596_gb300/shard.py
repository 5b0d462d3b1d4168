"""Host-side logic for running the bulb-model step on several GPUs, one process per GPU.

The paper distributes the angle bins of one problem over MPI ranks and sums the angular integrals
with one all-reduce per evaluation of the right-hand side (Sec. 3.3).  Here the work splits in
one of two ways:

* independent instances (a batch of problems): each rank takes whole instances and nothing is
  exchanged (``instance_shards``);
* one problem: each rank takes a contiguous range of the beam index (``beam_shards``); every
  integrator stage needs the moments of all beams, so the ranks exchange their partial moments
  once per stage (``allreduce_fixed``); ``evolve_sharded`` drives a beam-shard handle of the
  library pass by pass with that exchange (``exchange_words``).

The exchange is exact and deterministic: a partial moment is carried as the FP64 device
accumulators' own 128-bit fixed-point pair (hi 2^64 + lo = trunc(x 2^64), lo an unsigned and hi a
signed 64-bit word); ranks all-gather the pairs and add them as exact integers, so the total does
not depend on the number of ranks, their order or the shard boundaries.
"""
from __future__ import annotations

import math

TWO64 = 1 << 64


def beam_shards(n_beams: int, world: int, align: int = 128):
    """Contiguous [lo, hi) ranges of the beam index, one per rank, boundaries on multiples of
    `align` (whole warps of a block), the last range taking the remainder."""
    if world < 1 or n_beams < 0:
        raise ValueError("need world >= 1 and n_beams >= 0")
    out = []
    for r in range(world):
        lo = (n_beams * r // world) // align * align
        hi = n_beams if r == world - 1 else (n_beams * (r + 1) // world) // align * align
        out.append((lo, max(lo, hi)))
    return out


def instance_shards(n_beams_per_instance, world: int):
    """Assign whole instances to ranks: largest first, each to the least-loaded rank (ties: the
    lowest rank).  Returns one sorted list of instance indices per rank."""
    load = [0] * world
    parts = [[] for _ in range(world)]
    order = sorted(range(len(n_beams_per_instance)), key=lambda i: (-n_beams_per_instance[i], i))
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += n_beams_per_instance[i]
    return [sorted(p) for p in parts]


def to_fixed(x: float):
    """(lo, hi) with hi 2^64 + lo = trunc(x 2^64), as the device accumulates: the split is taken
    on |x| (where |x| - floor(|x|) is exact) and negated as a 128-bit integer for x < 0."""
    if not math.isfinite(x):
        raise ValueError("non-finite moment")
    ax = abs(x)
    hi = math.floor(ax)
    lo = int((ax - hi) * 18446744073709551616.0)
    if x < 0:
        t = -(hi * TWO64 + lo)
        return t % TWO64, t // TWO64
    return lo, hi


def fixed_add(a, b):
    """Exact sum of two (lo, hi) pairs with the carry of the low word."""
    t = (a[1] * TWO64 + a[0]) + (b[1] * TWO64 + b[0])
    return t % TWO64, t // TWO64


def from_fixed(p) -> float:
    """The device's read-out: (double) hi + (double) lo * 2^-64."""
    return float(p[1]) + float(p[0]) * 5.421010862427522e-20


def _words_to_tensor(pairs, torch):
    # lo as the bit pattern of a signed 64-bit integer, hi as is
    flat = []
    for lo, hi in pairs:
        flat += [lo - TWO64 if lo >= (1 << 63) else lo, hi]
    return torch.tensor(flat, dtype=torch.int64)


def allreduce_fixed(pairs, group=None):
    """Exact all-reduce of a list of fixed-point pairs across the ranks of `group`
    (torch.distributed, any backend): all-gather every rank's words, then add them as integers
    in rank order.  Every rank returns the same list of pairs."""
    import torch
    import torch.distributed as dist

    mine = _words_to_tensor(pairs, torch)
    world = dist.get_world_size(group)
    if dist.get_backend(group) == "nccl":
        mine = mine.cuda()
    bufs = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(bufs, mine, group=group)
    out = [(0, 0)] * len(pairs)
    for b in bufs:
        w = [int(v) for v in b.cpu().tolist()]
        for c in range(len(pairs)):
            lo = w[2 * c] % TWO64
            out[c] = fixed_add(out[c], (lo, w[2 * c + 1]))
    return out


def max_over_ranks(x: float, group=None) -> float:
    """The largest value of x over the ranks (the benchmark's time of a step is the slowest
    rank's); x itself with no process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return x
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sum_words(parts):
    """Totals of the beam-shard word vectors of xflat_shard_partials: the (lo, hi) fixed-point
    pairs added exactly, the error maxima (bit patterns of non-negative doubles) by maximum, the
    non-finite flags by logical or."""
    n = len(parts[0])
    nm = (n - 2) // 2
    out = [0] * n
    for c in range(nm):
        t = 0
        for w in parts:
            t += (int(w[2 * c + 1]) << 64) + (int(w[2 * c]) % TWO64)
        lo = t % TWO64
        out[2 * c] = lo - TWO64 if lo >= (1 << 63) else lo
        out[2 * c + 1] = t >> 64
    out[2 * nm] = max(int(w[2 * nm]) for w in parts)
    out[2 * nm + 1] = 1 if any(int(w[2 * nm + 1]) for w in parts) else 0
    return out


def exchange_words(words, group=None):
    """All-gather this rank's word vector over `group` (torch.distributed, any backend) and return
    the totals (sum_words over the ranks in rank order: the same on every rank)."""
    import torch
    import torch.distributed as dist

    mine = torch.tensor([int(v) for v in words], dtype=torch.int64)
    if dist.get_backend(group) == "nccl":
        mine = mine.cuda()
    bufs = [torch.empty_like(mine) for _ in range(dist.get_world_size(group))]
    dist.all_gather(bufs, mine, group=group)
    return sum_words([b.cpu().tolist() for b in bufs])


def evolve_sharded(shards, r1, exchange=None):
    """Integrate one problem to r1 with beam-shard handles (objects with the Solver shard_* calls):
    `shards` is this process's handles (one per rank on several GPUs; several in one process to
    emulate ranks on one device), `exchange(word vector) -> totals` the cross-process reduction of
    this process's total (e.g. exchange_words; None: only the handles given).  Every pass runs on
    every shard before the exchange, so no kernel ever waits for another.  Returns the number of
    radial steps taken."""
    def reduce(ws):
        local = sum_words(ws)
        return exchange(local) if exchange is not None else local

    passes = shards[0].shard_info()[0]
    for s in shards:
        s.shard_begin(r1)
    for s in shards:
        s.shard_pass(-1)
    tot = reduce([s.shard_partials() for s in shards])
    done = False
    for s in shards:
        s.shard_set_totals(tot)
        done = s.shard_serial(True)
    steps = 0
    while not done:
        for p in range(passes):
            for s in shards:
                s.shard_pass(p)
            tot = reduce([s.shard_partials() for s in shards])
            for s in shards:
                s.shard_set_totals(tot)
        for s in shards:
            done = s.shard_serial(False)
        steps += 1
    return steps
