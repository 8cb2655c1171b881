"""The weak-scaling path of bench.py on two gloo ranks (CPU): environments are sharded by
seed with no data exchange, and only the timing is reduced (max time, summed work)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seeds = []
    for make in (bench.highspeed_workload, bench.config2_workload):   # both sharded lines
        w = make(4, rank)
        seeds.append([l.seed for e in w.envs for l in e.layers])
    t, units, events = bench.reduce_over_ranks(10.0 + rank, 1000 * (rank + 1), 7, "cpu")
    q.put((rank, seeds, t, units, events))
    dist.destroy_process_group()


def test_two_rank_sharding_and_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, t0, u0, e0), (r1, s1, t1, u1, e1) = out
    for a, b in zip(s0, s1):
        assert not set(a) & set(b)              # disjoint scenes per rank
    assert t0 == t1 == 11.0                     # slowest rank's time
    assert u0 == u1 == 3000 and e0 == e1 == 14  # work summed over ranks


def test_e2e_leg_stays_inside_its_share_of_host_memory(monkeypatch):
    """The end-to-end leg pins at most 0.6 of the host's available memory divided by the
    ranks: when two keyframes and the event buffer do not fit that share it reports why and
    pins nothing (no CUDA call is made on that path)."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    gib = 1 << 30
    monkeypatch.setattr(bench, "host_mem_available", lambda: 100 * gib)

    class Plane:                      # the leg reads only the element count of a keyframe
        def __init__(self, n):
            self.n = n

        def numel(self):
            return self.n

    kf = (Plane(gib // 4), Plane(2 * gib // 4), Plane(2 * gib // 4))   # 5 GiB of float32
    dev = [kf] * 7
    capacity = 10 * gib // 16                                       # a 10 GiB event buffer
    out = bench.e2e_leg(None, None, dev, 6, capacity, 0, dist=None, world=8)   # 7.5 GiB share
    assert "skipped" in out
    out = bench.e2e_leg(None, None, dev, 6, capacity, 0, dist=None, world=4)   # 15 GiB share: 0 gaps
    assert "skipped" in out


def test_link_floor_takes_the_slowest_bound():
    """The end-to-end leg's link floor: each direction at its own rate, both together at
    their summed rate (5 GB up and 15 GB down at 50 / 50 / 75 GB/s: the way down alone,
    0.3 s; 15 GB each way: the shared rate, 0.4 s)."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    r = {"h2d_gbs": 50.0, "d2h_gbs": 50.0, "both_gbs": 75.0}
    assert abs(bench.link_floor_ms(5e9, 15e9, r) - 300.0) < 1e-9
    assert abs(bench.link_floor_ms(15e9, 15e9, r) - 400.0) < 1e-9
    assert abs(bench.link_floor_ms(0, 0, r)) == 0.0


def test_e2e_slices_cover_every_environment_once():
    """The end-to-end leg's slices: consecutive, covering every environment once, each
    buffer at least its share of the capacity (with a margin that grows as slices shrink) and
    at most the whole; the planes' views of a slice hold exactly its environments' pixels."""
    import sys
    import numpy as np
    import torch
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    for n_env, S in ((1024, 4), (16, 4), (3, 4), (1, 4), (7, 1)):
        cut, caps = bench.slice_plan(n_env, S, 1_000_000)
        assert cut[0] == 0 and cut[-1] == n_env and len(caps) == len(cut) - 1 == min(S, n_env)
        assert all(cut[q] < cut[q + 1] for q in range(len(caps)))
        for q, c in enumerate(caps):
            share = 1_000_000 * (cut[q + 1] - cut[q]) / n_env
            assert (c >= 1.2 * share or c == 1_000_000) and c <= 1_000_000
    # three environments of 2, 3 and 4 pixels; planes of 1 and 2 values per pixel
    px = np.cumsum([0, 2, 3, 4])
    L = torch.arange(9, dtype=torch.float32)
    mv = torch.arange(18, dtype=torch.float32)
    a, b = bench.slice_planes((L, mv), px, 1, 3)
    assert a.tolist() == [2, 3, 4, 5, 6, 7, 8] and b.tolist() == list(range(4, 18))
    a, b = bench.slice_planes((L, mv), px, 0, 1)
    assert a.tolist() == [0, 1] and b.tolist() == [0, 1, 2, 3]
