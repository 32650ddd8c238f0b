"""Multi-rank path: world-size-2 gloo ranks split the triple loop by weight
and sum their partial results with all-reduce; the sum equals the unsharded
result.  On the CPU both ranks run the oracle; on a GPU both ranks drive the
library (shard.omega_sharded, host-pointer contexts on the same device, the
all-reduce over gloo on host copies)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from cc3_inputs import make_inputs
from paper_2007_01088_gb300.shard import triple_partition, triples_with_weights


def test_partition_covers_every_triple_once_and_balances():
    for no in (1, 2, 5, 16):
        for world in (1, 2, 3, 8):
            parts = [triple_partition(no, world, r) for r in range(world)]
            flat = [t for p in parts for t in p]
            all_t = [t for t, _ in triples_with_weights(no)]
            assert sorted(flat) == sorted(all_t) and len(flat) == len(set(flat))
            w = dict(triples_with_weights(no))
            loads = [sum(w[t] for t in p) for p in parts]
            if loads and max(loads) > 0:
                assert max(loads) - min(loads) <= 6


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        inp = make_inputs(5, 12, seed=3)
        part = triple_partition(inp.no, world, rank)
        r = oracle.omega_inputs(inp, triples=part, nthreads=1)
        o1 = torch.from_numpy(r["omega1"].copy())
        o2 = torch.from_numpy(r["omega2"].copy())
        e = torch.tensor([r["E_T"]], dtype=torch.float64)
        for x in (o1, o2, e):
            dist.all_reduce(x)
        if rank == 0:
            full = oracle.omega_inputs(inp, nthreads=1)
            q.put((float(np.abs(o1.numpy() - full["omega1"]).max()),
                   float(np.abs(o2.numpy() - full["omega2"]).max()),
                   abs(float(e[0]) - full["E_T"])))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_to_full_result():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    d1, d2, de = q.get(timeout=10)
    assert d1 <= 1e-14 and d2 <= 1e-14 and de <= 1e-12


def _lib_rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_2007_01088_gb300 as g
        from paper_2007_01088_gb300.shard import omega_sharded
        inp = make_inputs(6, 40, seed=8)
        ctx = g.Context(inp)
        for prec in (g.CC3_FP64, g.CC3_SPLIT_BF16):
            out = (torch.zeros((6, 40), dtype=torch.float64),
                   torch.zeros((6, 6, 40, 40), dtype=torch.float64),
                   torch.zeros((1,), dtype=torch.float64))
            omega_sharded(ctx, prec, out)
            if rank == 0:
                import oracle
                full = oracle.omega_inputs(inp)
                q.put((prec, float(np.abs(out[0].numpy() - full["omega1"]).max()),
                       float(np.abs(out[1].numpy() - full["omega2"]).max()),
                       abs(float(out[2][0]) - full["E_T"]),
                       float(np.abs(full["omega2"]).max()), abs(full["E_T"])))
        ctx.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
def test_two_gloo_ranks_drive_the_library_and_sum_to_full_result():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_lib_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=600)
        assert p.exitcode == 0
    for _ in range(2):
        prec, d1, d2, de, m2, me = q.get(timeout=10)
        if prec == 0:  # FP64: 1e-12 relative
            assert d2 <= 1e-12 * m2 and de <= 1e-12 * me
        else:          # split: 1e-9 absolute and 1e-10 relative
            assert d2 <= min(1e-9, 1e-10 * m2) and de <= min(1e-8, 1e-10 * me)
