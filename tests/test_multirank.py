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
