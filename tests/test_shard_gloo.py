"""Multi-rank path on CPU: world_size 2 gloo ranks split the pairs of one
workload, compute them with the oracle, and rank 0 gathers H and S."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2404_10223_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out, fail_rank):
    import torch.distributed as dist
    from oracle import mps as om
    from paper_2404_10223_gb300 import inputs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import datetime
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    try:
        w = inputs.workload("n6_chi8")
        pairs = w.all_pairs()
        o = om.Context(w.h1, w.eri, w.N, w.n_alpha, w.n_beta)
        for m in w.mps:
            o.add_mps(m.tensors, m.U)
        dims = [m.bond_dims for m in w.mps]
        mpo_dims = o.mpo(0).dims
        costs = [shard.pair_cost(dims[i], dims[j], mpo_dims, i == j) for i, j in pairs]
        parts = shard.partition_pairs(pairs, costs, world)
        if rank == fail_rank:
            raise RuntimeError("injected failure before the exchange")
        local = {}
        for k in parts[rank]:
            i, j = pairs[k]
            h, s, _ = o.pair(i, j)
            local[(i, j)] = (h, s)
        H, S = shard.gather_to_root(local, w.M, rank, world)
        if rank == 0:
            out.put(("ok", H.tolist(), S.tolist(), [len(p) for p in parts]))
    except Exception as e:  # reported to the parent
        out.put(("error", rank, repr(e)))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def test_partition_balances_and_covers():
    costs = [5.0, 1.0, 1.0, 1.0, 3.0, 2.0, 2.0]
    pairs = [(0, k) for k in range(len(costs))]
    parts = shard.partition_pairs(pairs, costs, 2)
    assert sorted(parts[0] + parts[1]) == list(range(len(costs)))
    loads = [sum(costs[k] for k in p) for p in parts]
    assert max(loads) - min(loads) <= max(costs)


def test_two_gloo_ranks_match_single_process():
    from oracle import mps as om
    from paper_2404_10223_gb300 import inputs
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q, -1)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert res[0] == "ok", res
    H, S = np.array(res[1]), np.array(res[2])
    assert min(res[3]) >= 1
    w = inputs.workload("n6_chi8")
    o = om.Context(w.h1, w.eri, w.N, w.n_alpha, w.n_beta)
    for m in w.mps:
        o.add_mps(m.tensors, m.U)
    for i, j in w.all_pairs():
        h, s, _ = o.pair(i, j)
        assert abs(H[i, j] - h) < 1e-12 and abs(S[i, j] - s) < 1e-12


def test_failed_rank_is_reported_not_hung():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q, 1)) for r in range(2)]
    for p in procs:
        p.start()
    msgs = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
    assert any(m[0] == "error" and m[1] == 1 and "injected" in m[2] for m in msgs)
    assert all(m[0] == "error" for m in msgs)          # rank 0 learns of it: its gather fails
