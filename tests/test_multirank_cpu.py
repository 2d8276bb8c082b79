"""Multi-rank host logic on CPU (gloo, world size 2): replica sharding and the final
argmin exchange.  Each rank anneals its shard with the oracle (standing in for its GPU);
the global result must equal the best over the union of both shards, and the union of
shards must be the single-rank run."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2407_10205_gb300.multigpu import shard


def test_shard_covers_every_replica_once():
    for total in (1, 7, 256, 1023):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                a, n = shard(total, world, r)
                seen.extend(range(a, a + n))
            assert seen == list(range(total))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_q):
    import torch.distributed as dist
    import oracle
    from paper_2407_10205_gb300 import instances as ins
    from paper_2407_10205_gb300.multigpu import global_best, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d = ins.sk_pm1(20, 3)
    P = oracle.Instance(d.kh, k=d.k)
    first, count = shard(12, world, rank)
    res = oracle.anneal(P, count, 150, 9, 0, 0.05, 2.0, 0.2, 2.0, r0=first, threads=1)
    k = int(np.lexsort((res["best_step"], res["best_e"]))[0])
    e, s, winner, spins = global_best(int(res["best_e"][k]), int(res["best_step"][k]), res["best_s"][k])
    out_q.put((rank, e, s, winner, spins, res["best_e"].tolist(), first))
    dist.destroy_process_group()


def test_two_ranks_agree_with_one_rank():
    import oracle
    from paper_2407_10205_gb300 import instances as ins
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    outs = sorted([q.get(timeout=120) for _ in range(2)], key=lambda o: o[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks hold the same global result
    assert outs[0][1:4] == outs[1][1:4] and np.array_equal(outs[0][4], outs[1][4])
    # it is the best of one rank-free run over all 12 replicas
    d = ins.sk_pm1(20, 3)
    P = oracle.Instance(d.kh, k=d.k)
    full = oracle.anneal(P, 12, 150, 9, 0, 0.05, 2.0, 0.2, 2.0, threads=1)
    assert sorted(outs[0][5] + outs[1][5]) == sorted(full["best_e"].tolist())
    e = outs[0][1]
    assert e == full["best_e"].min()
    assert oracle.energy_exact(P, outs[0][4]) == e
