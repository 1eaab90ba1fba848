"""G4 partitioned over ranks (Sec. 3.1, Algorithms 1-2), host side, on CPU:
the partition plan, and runs of 2 and 4 gloo ranks whose device work is the
CPU oracle restricted to each rank's slab of transfer frequencies; the slabs,
put together, equal the single-process oracle result."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2105_00027_gb300 import inputs, shard

P = inputs.Problem


def test_plan_covers_every_m_and_measurement_once():
    for world in (1, 2, 3, 4, 6, 8):
        for Nwex in (1, 2, 3, 4, 5, 8):
            s, g = shard.plan(world, Nwex)
            assert s * g == world and 1 <= s <= Nwex
            ms = []
            for j in range(s):
                first, count = shard.slab(j, s, Nwex)
                assert count >= 1
                ms += list(range(first, first + count))
            assert ms == list(range(Nwex))
            R, batch = 29, 4
            seen = []
            for rank in range(world):
                lay = shard.layout(rank, world, Nwex)
                rounds = shard.measurements_of(lay, R, batch)
                if lay.shard == 0:
                    for block, _ in rounds:
                        seen += block
                # inside a group the shards contribute disjoint parts of each block
                for block, mine in rounds:
                    assert set(mine) <= set(block)
            assert sorted(seen) == list(range(R))
    with pytest.raises(ValueError):
        shard.plan(4, 2, shards=3)


class OracleEngine:
    """The CPU oracle as a rank's device: the unnormalised sum over the
    measurements it is handed, on the rank's slabs (every q, its m)."""

    def __init__(self, p, m_first, m_count):
        self.p = p
        self.d = oracle.dims(p.Lx, p.Ly, p.Nw, p.Nwex, p.Nkex)
        q, m = np.meshgrid(np.arange(p.Nkex), np.arange(m_first, m_first + m_count), indexing="ij")
        self.qsel = q.ravel().astype(np.int32)
        self.msel = m.ravel().astype(np.int32)
        self.acc = np.zeros((len(self.qsel), p.Nw2, p.Nw2, p.Nc, p.Nc), np.complex128)
        self.S = 0.0
        self.G0 = inputs.g0(p)

    def stage(self, M, s):
        Mn = M.numpy()
        Gu = oracle.build_G(Mn[0], self.G0[0])
        Gd = oracle.build_G(Mn[1], self.G0[1])
        oracle.accumulate(self.d, Gu, Gd, s, self.acc, self.qsel, self.msel, nthreads=1)
        self.S += s

    def result(self):
        import torch
        return torch.from_numpy(self.acc.copy()), self.S


def _rank_main(rank, world, port, p, shards, outdir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lay = shard.layout(rank, world, p.Nwex, shards)
    gpg, cpg = shard.ShardedRun.process_groups(dist, lay)
    run = shard.ShardedRun(lay, dist, gpg, cpg)
    signs = inputs.signs(p, seed=4)
    eng = OracleEngine(p, lay.m_first, lay.m_count)
    slab_t, S = run.run(eng, p.R, p.batch, lambda r: inputs.measurement_M(p, r, seed=4),
                        lambda r: signs[r])
    np.save(os.path.join(outdir, "rank%d.npy" % rank), slab_t.numpy())
    np.save(os.path.join(outdir, "rank%d_S.npy" % rank), np.array([S, lay.m_first, lay.m_count]))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,shards", [(2, 2), (4, 2)])
def test_ranks_gloo_match_single_oracle(world, shards, tmp_path):
    import torch.multiprocessing as mp
    p = P(2, 2, 4, 4, 4, 5.0, 21, 4)
    mp.spawn(_rank_main, args=(world, _free_port(), p, shards, str(tmp_path)), nprocs=world)
    d = oracle.dims(p.Lx, p.Ly, p.Nw, p.Nwex, p.Nkex)
    signs = inputs.signs(p, seed=4)
    M = inputs.batch_M(p, 0, p.R, seed=4).numpy()
    ref, Sref = oracle.run(d, M, inputs.g0(p), signs)            # every (q, m), q-major
    ref = ref.reshape(p.Nkex, p.Nwex, p.Nw2, p.Nw2, p.Nc, p.Nc)
    covered = np.zeros(p.Nwex, int)
    for rank in range(world):
        got = np.load(str(tmp_path / ("rank%d.npy" % rank)))
        S, first, count = np.load(str(tmp_path / ("rank%d_S.npy" % rank)))
        first, count = int(first), int(count)
        assert S == Sref
        want = ref[:, first:first + count].reshape(got.shape)
        err = oracle.errors(want, got)
        assert err["L2"] <= 1e-13, (rank, err)
        if rank < shards:
            covered[first:first + count] += 1
    assert np.all(covered == 1)
