"""Host-side logic of the replica (N > 1) benchmark path, run as two gloo ranks
on the CPU: distinct cubes per rank, the timing barrier, the max over ranks,
and rank-0-only reporting of the reference arm."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        seed = bench.replica_seed(2, r)
        bench.barrier(w)
        m = bench.max_over_ranks(float(10 * (r + 1)), w)
        # the reference arm reports on rank 0 only
        args = type("A", (), {"steps": 1, "warmup": 0, "cpu_budget": 0.0, "tucker": 0,
                              "precision": "auto"})()
        ref = bench.run_reference(args, "c1")
        q.put((r, w, local, seed, m, ref is None))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    (r0, w0, l0, s0, m0, none0), (r1, w1, l1, s1, m1, none1) = got
    assert (r0, r1) == (0, 1) and w0 == w1 == 2 and (l0, l1) == (0, 1)
    assert s0 != s1                      # each replica denoises its own cube
    assert m0 == m1 == 20.0              # max over ranks seen by every rank
    assert not none0 and none1           # only rank 0 prints the reference line


def test_single_rank_defaults(monkeypatch):
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 1, 0)
    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)


def test_kernel_work_table():
    import bench
    kind, b = bench.kernel_work("fs_dual", (200, 200, 80))
    assert kind == "hbm" and b == 23 * 4 * 3_200_000
    kind, f = bench.kernel_work("cgemm_e", (200, 200, 80))
    assert kind == "alu" and f == 8 * 200 * 200 * 200 * 3 * 41
