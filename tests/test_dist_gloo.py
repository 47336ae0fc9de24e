"""Two CPU ranks (gloo) each step their own shard of cells with the oracle and
sum the tally: identical to one process stepping every cell, because cells
are independent and keyed by their global index."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2604_24627_gb300 import dist as pdist  # noqa: E402

NCELLS = 10


def _tally_of(cells):
    from oracle import step as ostep, tally as otally
    from oracle.plasma import Params
    p = Params(g_agg_GeV_inv=1e-10, g_ae=2e-12, dt_phys_s=2e12, w_a=3e9, seed=21)
    H = np.zeros((3, 160))
    tot = {"events": 0.0, "dE": 0.0}
    for c in cells:
        parts = ostep.init_cell(p, c, 3.0, 6e25, 1e-12, 24, 16, 4)
        ci = ostep.CellInput(3.0, np.array([6e25]), np.array([1.0]), np.array([1.00794]))
        t, fb = ostep.step_cell(ci, parts, p, 3, c, 7)
        n = len(t.new_axion_E)
        w_new = parts["a"].w[len(parts["a"]) - n:]
        for k, ch in enumerate((1, 2, 4)):
            sel = t.new_axion_channel == ch
            H[k] += otally.histogram(t.new_axion_E[sel], w_new[sel], 160, 80.0)
        tot["events"] += sum(t.events.values())
        tot["dE"] += t.dE
    return H, tot


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, count = pdist.shard_range(NCELLS, world, rank)
    H, tot = _tally_of(range(first, first + count))
    Hs, tots = pdist.allreduce_tally(H, tot, dist)
    if rank == 0:
        q.put((Hs, tots))
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_shard_range_partitions():
    for n in (0, 1, 7, 64, 65536):
        for world in (1, 2, 3, 8):
            got = [pdist.shard_range(n, world, r) for r in range(world)]
            assert sum(c for _, c in got) == n
            assert all(got[i][0] + got[i][1] == got[i + 1][0] for i in range(world - 1))
            assert max(c for _, c in got) - min(c for _, c in got) <= 1


def test_two_gloo_ranks_equal_one_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    Hs, tots = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    H1, tot1 = _tally_of(range(NCELLS))
    np.testing.assert_allclose(Hs, H1, rtol=1e-12, atol=0)
    assert tots["events"] == tot1["events"] > 0
    assert abs(tots["dE"] - tot1["dE"]) <= 1e-9 * abs(tot1["dE"])
