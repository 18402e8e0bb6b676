"""Multi-rank path on CPU (gloo, world size 2): shift sharding and the
final two-step average (Eq. 9, Sec. II.B step 4) across ranks equal the
single-process average.  The per-shift currents come from the oracle."""
import os
import socket

import numpy as np
import pytest

import workloads as W
from oracle import dynamics, kpoints
from oracle.cell import Grid


def test_shard_ranges_balanced_and_complete():
    from paper_2112_00920_gb300.distributed import shard_ranges
    costs = [5, 1, 1, 1, 8, 2, 2, 4]
    for world in (1, 2, 3, 4, 8, 10):
        r = shard_ranges(costs, world)
        assert len(r) == world
        assert r[0][0] == 0 and r[-1][1] == len(costs)
        assert all(a[1] == b[0] for a, b in zip(r[:-1], r[1:]))
    r2 = shard_ranges([1.0] * 64, 2)
    assert r2 == [(0, 32), (32, 64)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _per_shift_dj():
    cell = W.cell_tiny(atoms="pair", n=(8, 8, 8), a=(6.0, 6.0, 6.0), n_bands=2)
    g = Grid(cell)
    out = []
    for i, s in enumerate(W.lattice_shifts(2)[:5]):
        k = kpoints.kpoints_cartesian(cell.a, (1, 1, 1), s)
        psi = W.random_orbitals(1, 2, cell.n, g.dv, seed=30, tag=i)
        r = dynamics.propagate(cell, k, psi, 0.08, 3, dynamics.field_samples(W.Kick(k0=0.01), 0.08, 3),
                               keep_state=False)
        out.append(r["J"] - r["J0_minus"][None, :])
    return np.stack(out)


def _worker(rank, world, port, dj_all, q):
    import torch.distributed as dist
    from paper_2112_00920_gb300.distributed import run_sharded
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seen = []

    def run_block(b, e):
        # the benchmark propagates its block through the library here; the test
        # takes the oracle's per-shift currents of the block
        seen.append((b, e))
        return dj_all[b:e].sum(axis=0)

    avg, block = run_sharded([1.0] * dj_all.shape[0], run_block)
    assert seen == [block]
    q.put((rank, avg, block))
    dist.destroy_process_group()


def test_two_step_average_across_two_gloo_ranks():
    import torch.multiprocessing as mp
    dj_all = _per_shift_dj()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, dj_all, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = dj_all.mean(axis=0)
    blocks = sorted(r[2] for r in res)
    assert blocks[0][0] == 0 and blocks[0][1] == blocks[1][0] and blocks[1][1] == dj_all.shape[0]
    for _, avg, _ in res:
        np.testing.assert_allclose(avg, ref, rtol=0, atol=1e-15 * np.max(np.abs(ref)) + 1e-20)
