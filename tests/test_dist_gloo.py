"""The multi-rank path on CPU: two gloo ranks, each stepping its own shard of
envs (the oracle stands in for the GPU), with the id offsets and the timing
reduction that bench.py uses under torchrun.

Checked: each rank's ids follow the previous rank's; a rank's outputs equal
a single process stepping the same envs with the same global ids; the two
shards have identical clean readings (same geometry) but independent dead
masks and noise (distinct ids); the max-over-ranks reduction.
"""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shard_outputs(gid0, egid0):
    import oracle
    from paper_2606_22332_gb300 import workload as W
    from _scenes import oracle_objects

    wl = W.config0(n_envs=4)
    wl.params = dict(wl.params, p_dead=0.2)
    geom = wl.geom()
    geom["taxel_gid0"] = geom["taxel_gid0"] + gid0
    geom["env_gid"] = geom["env_gid"] + egid0
    osc = oracle.OracleScene(geom, oracle_objects(wl.objects, wl.params), wl.params)
    st = osc.new_state()
    osc.reset(st, 0)
    outs = [osc.step(st, wl.inputs(s)) for s in range(2)]
    o = outs[-1]
    return np.concatenate([o["depth_clean"], o["depth_noisy"], o["ft_clean"].ravel(), o["ft_noisy"].ravel(),
                           st["flags"].astype(np.float64)]), wl.n_envs, wl.n_taxels


def _worker(rank, world, port, q):
    sys.path[:0] = [ROOT, HERE]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    from paper_2606_22332_gb300 import dist as D

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = D.rank_env()
    from paper_2606_22332_gb300 import workload as W

    wl = W.config0(n_envs=4)
    gid0, egid0 = D.shard_ids(r, wl.n_envs, wl.n_taxels)
    vec, _, _ = _shard_outputs(gid0, egid0)
    t = torch.tensor(vec)
    got = [torch.zeros_like(t) for _ in range(ws)]
    dist.all_gather(got, t)
    tmax = D.max_over_ranks(10.0 + r)
    if r == 0:
        q.put({"ws": ws, "local": local, "ids": (gid0, egid0), "tmax": tmax, "vecs": [g.numpy() for g in got]})
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_step_their_own_shards():
    import oracle
    from paper_2606_22332_gb300 import dist as D
    from paper_2606_22332_gb300 import workload as W

    oracle.build()
    wl = W.config0(n_envs=4)
    E, T = wl.n_envs, wl.n_taxels
    assert D.shard_ids(0, E, T) == (0, 0) and D.shard_ids(1, E, T) == (T, E) and D.shard_ids(3, E, T) == (3 * T, 3 * E)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=240)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert res["ws"] == 2 and res["local"] == 0 and res["tmax"] == 11.0
    v0, v1 = res["vecs"]
    # each rank equals one process stepping the same envs with the same global ids
    s0, _, _ = _shard_outputs(0, 0)
    s1, _, _ = _shard_outputs(T, E)
    assert np.array_equal(v0, s0) and np.array_equal(v1, s1)
    # same geometry, distinct ids: equal clean depths, independent dead masks and noise
    assert np.array_equal(v0[:T], v1[:T])
    flags0, flags1 = v0[-T:].astype(np.uint8), v1[-T:].astype(np.uint8)
    assert not np.array_equal((flags0 >> 1) & 1, (flags1 >> 1) & 1)
    assert not np.array_equal(v0[T:2 * T], v1[T:2 * T])
