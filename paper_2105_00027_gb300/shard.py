"""G4 partitioned over several GPUs, every measurement seen by every rank.

The paper distributes G_t (G4) so that each of p ranks holds 1/p of it
(Sec. 3.1) and passes every walker's G_sigma around a ring so that each rank
adds every measurement to its own part (Algorithm 1); ranks can also form
sub-rings that split the measurements and sum their parts at the end
(Sec. 3.2.1, Algorithm 2).  Here:

* a rank's part is a slab of the bosonic transfer frequencies m (all momenta
  q): the handle option ``wex_slab`` (``options.wex_first/wex_count`` in the C
  ABI), whose exported array is a contiguous block of planes of the whole
  problem's export;
* the ranks form ``groups`` of ``shards`` ranks; inside a group the shards
  hold disjoint slabs that together cover every m, and per batch round they
  all-gather the M matrices (and signs) of their measurements, so that each
  shard stages the whole batch -- the collective that takes the place of the
  ring;
* the groups split the run's measurements between them (the sub-rings); at
  the end the unnormalised slabs and sign sums of the ranks holding the same
  slab are summed (all-reduce) before the division by the sign sum.

The device work of a rank is whatever ``engine`` does with the measurements it
is handed (the library's handle on a GPU; the tests pass the CPU oracle on
gloo ranks).  This module only plans the partition and moves data.
"""
from __future__ import annotations

import math
from dataclasses import dataclass


@dataclass(frozen=True)
class Layout:
    """Where rank `rank` of `world` sits: its group, its shard in the group and
    its slab of transfer frequencies [m_first, m_first + m_count)."""
    world: int
    shards: int
    groups: int
    rank: int
    group: int
    shard: int
    m_first: int
    m_count: int


def plan(world: int, Nwex: int, shards: int = 0):
    """(shards, groups): the largest divisor of `world` not above Nwex as the
    number of slabs (every slab holds at least one m), unless `shards` is
    given."""
    if shards <= 0:
        shards = max(s for s in range(1, min(world, Nwex) + 1) if world % s == 0)
    if world % shards or shards > Nwex:
        raise ValueError("shards must divide the world size and not exceed Nwex")
    return shards, world // shards


def slab(shard: int, shards: int, Nwex: int):
    """Contiguous, as even as possible: (first m, count)."""
    base, extra = divmod(Nwex, shards)
    first = shard * base + min(shard, extra)
    return first, base + (1 if shard < extra else 0)


def layout(rank: int, world: int, Nwex: int, shards: int = 0) -> Layout:
    s, g = plan(world, Nwex, shards)
    group, shard = divmod(rank, s)
    first, count = slab(shard, s, Nwex)
    return Layout(world, s, g, rank, group, shard, first, count)


def measurements_of(lay: Layout, R: int, batch: int):
    """The run's measurement indices handled by this rank's group, as batch
    rounds: round b of group g is the g-th block of `batch` indices of
    super-round b (the groups take consecutive blocks), and inside a round
    shard j contributes the indices j, j + shards, ... of the block."""
    rounds = []
    per = batch * lay.groups
    for start in range(0, R, per):
        b0 = start + lay.group * batch
        block = list(range(b0, min(R, b0 + batch)))
        rounds.append((block, block[lay.shard::lay.shards]))
    return rounds


class ShardedRun:
    """Drives one rank of a partitioned run.

    engine: stage(M, sign) for every measurement of the group (its own and the
    gathered ones, in the group's order), result() -> (unnormalised slab as a
    tensor, sign sum) at the end.  get_M(r) -> the rank's M of measurement r as
    a tensor [2][N][N] (complex) on the collective's device; sign(r) -> s_r.
    """

    def __init__(self, lay: Layout, dist, group_pg=None, column_pg=None):
        self.lay = lay
        self.dist = dist
        self.group_pg = group_pg
        self.column_pg = column_pg

    @staticmethod
    def process_groups(dist, lay: Layout):
        """Create (every rank, in the same order) the groups' and the slab
        columns' process groups; returns this rank's (group, column)."""
        mine_g = mine_c = None
        for g in range(lay.groups):
            pg = dist.new_group(list(range(g * lay.shards, (g + 1) * lay.shards)))
            if g == lay.group:
                mine_g = pg
        for j in range(lay.shards):
            pg = dist.new_group([g * lay.shards + j for g in range(lay.groups)])
            if j == lay.shard:
                mine_c = pg
        return mine_g, mine_c

    def gather_round(self, block, mine, get_M, sign, chunk=8):
        """All-gather the M (and signs) of one round inside the group, `chunk`
        measurements per shard at a time (bounded buffers); yields (M, s) for
        every index of `block`, in block order."""
        import torch
        lay = self.lay
        if lay.shards == 1:
            for r in block:
                yield get_M(r), float(sign(r))
            return
        shape = M0 = None
        for c0 in range(0, math.ceil(len(block) / lay.shards), chunk):
            sub = block[c0 * lay.shards:(c0 + chunk) * lay.shards]
            mine_sub = sub[lay.shard::lay.shards]
            per = math.ceil(len(sub) / lay.shards)
            if M0 is None:
                # the shape, type and device of M (a shard without a measurement
                # in a ragged chunk still takes part; its slots carry zeros)
                M0 = get_M(sub[0])
                shape, dtype, device = tuple(M0.shape), M0.dtype, M0.device
            send = torch.zeros((per,) + shape, dtype=dtype, device=device)
            for i, r in enumerate(mine_sub):
                send[i] = get_M(r)
            sig = torch.tensor([float(sign(r)) for r in mine_sub] + [0.0] * (per - len(mine_sub)),
                               dtype=torch.float64, device=device)
            recv = torch.empty((lay.shards * per,) + shape, dtype=dtype, device=device)
            rsig = torch.empty(lay.shards * per, dtype=torch.float64, device=device)
            real_send = torch.view_as_real(send) if send.is_complex() else send
            real_recv = torch.view_as_real(recv) if recv.is_complex() else recv
            self.dist.all_gather_into_tensor(real_recv, real_send, group=self.group_pg)
            self.dist.all_gather_into_tensor(rsig, sig, group=self.group_pg)
            signs = rsig.cpu().tolist()
            for idx in range(len(sub)):
                j, i = idx % lay.shards, idx // lay.shards   # shard j's i-th measurement
                yield recv[j * per + i], signs[j * per + i]

    def run(self, engine, R, batch, get_M, sign):
        for block, mine in measurements_of(self.lay, R, batch):
            for M, s in self.gather_round(block, mine, get_M, sign):
                engine.stage(M, s)
        return self.finish(engine)

    def finish(self, engine):
        """Sum the slabs and sign sums of the ranks holding the same slab and
        normalise: (slab / sum of signs, sum of signs)."""
        import torch
        acc, S = engine.result()
        if self.lay.groups > 1:
            real = torch.view_as_real(acc) if acc.is_complex() else acc
            self.dist.all_reduce(real, group=self.column_pg)
            t = torch.tensor([S], dtype=torch.float64, device=acc.device)
            self.dist.all_reduce(t, group=self.column_pg)
            S = float(t.item())
        if S != 0.0:
            acc.div_(S)
        return acc, S


class HandleEngine:
    """A rank's G4 slab on its GPU: the library's handle with
    ``wex_slab = (m_first, m_count)``.  result() finalises into `out` (the
    slab in the exported order) and returns it unnormalised with the sign
    sum, for the sum over groups."""

    def __init__(self, handle, G0, out=None):
        self.h = handle
        self.G0 = G0
        self.out = out

    def stage(self, M, sign):
        self.h.compute_G(M, self.G0, sign)

    def result(self):
        out, S = self.h.finalize(self.out, allow_zero_sign=True)
        if S != 0.0:
            out.mul_(S)   # in place: the slab can be tens of GB
        return out, S
