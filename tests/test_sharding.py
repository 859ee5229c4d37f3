"""Multi-rank host logic on CPU: source partition and the J^T sum over ranks, run as
world-size-2 gloo process groups (the GPU pool gives one device per call)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2609_14982_b300.sharding import partition_sources, source_cost


def test_partition_is_balanced_and_complete():
    costs = [source_cost(1000, L, 8) for L in (10, 40, 30, 20, 25, 5, 35)]
    parts = partition_sources(costs, 3)
    flat = sorted(a for p in parts for a in p)
    assert flat == list(range(7))
    loads = [sum(costs[a] for a in p) for p in parts]
    assert max(loads) - min(loads) <= max(costs)
    assert partition_sources(costs, 3) == parts          # deterministic
    assert partition_sources([1.0], 4)[0] == [0]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, case, q):
    import torch
    import torch.distributed as dist

    import oracle as O
    from paper_2609_14982_b300.sharding import partition_sources, reduce_model_gradient
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g, Ts, s, srcs, rec, p, y = case
    _, G, _ = O.metric(g)
    parts = partition_sources([1.0 + a for a in range(len(srcs))], world)
    mine = parts[rank]
    tans = [O.build_tangent(g, G, Ts[a], s, int(srcs[a])) for a in mine]
    # J: each rank's rows, no exchange
    jp = O.J(tans, s, rec, p) if mine else np.zeros((0, len(rec), p.shape[1]))
    # J^T: partial sum over own sources, then one all-reduce
    part = O.JT(tans, s, rec, y[mine]) if mine else np.zeros((g.N, p.shape[1]))
    t = torch.tensor(part)
    reduce_model_gradient(t)
    q.put((rank, mine, jp, t.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_jacobian_actions_gloo(oracle_mod):
    from paper_2609_14982_b300 import workloads as W
    wl = W.config1()
    g = wl.grid
    srcs = np.array([wl.src[0], g.index(30, 0), g.index(45, 0)], dtype=np.int32)
    s = 1.0 / (1.5 + 0.5 * g.xyz[:, 1])
    Ts = np.stack([W.linear_velocity_T(g.xyz, g.xyz[k], 1.5, 0.5) for k in srcs])
    rng = np.random.default_rng(9)
    p = rng.standard_normal((g.N, 2))
    y = rng.standard_normal((len(srcs), len(wl.rec), 2))
    case = (g, Ts, s, srcs, wl.rec, p, y)
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = [q.get() for _ in range(world)]
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    _, G, _ = oracle_mod.metric(g)
    tans = [oracle_mod.build_tangent(g, G, Ts[a], s, int(srcs[a])) for a in range(len(srcs))]
    full_jp = oracle_mod.J(tans, s, wl.rec, p)
    full_jt = oracle_mod.JT(tans, s, wl.rec, y)
    for rank, mine, jp, jt in res:
        assert np.allclose(jt, full_jt, rtol=1e-13, atol=1e-13 * np.abs(full_jt).max())
        for k, a in enumerate(mine):
            assert np.array_equal(jp[k], full_jp[a])
    assert sorted(a for _, mine, _, _ in res for a in mine) == list(range(len(srcs)))
