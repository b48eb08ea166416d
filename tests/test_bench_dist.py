"""The N > 1 path of bench.py on the CPU: two gloo ranks (world size 2) run
the rank logic the GPU job uses -- each rank its own beam seed, the step
time taken as the maximum over ranks, the whole-job rate over all ranks'
solves -- and the reference arm leaves ranks other than 0 without work."""
import importlib.util
import multiprocessing as mp
import os
import socket

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    b = _bench()
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, local = b._dist()
        ms = 10.0 + 5.0 * r                       # rank 1 is the slower one
        step = b._max_over_ranks(ms, w, "cpu")
        out.put((r, w, local, b._rank_seed(r), step, b._job_rate(w, 64, step)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, s0, t0, v0), (r1, w1, l1, s1, t1, v1) = res
    assert (r0, r1) == (0, 1) and w0 == w1 == 2 and (l0, l1) == (0, 1)
    assert s0 != s1                                   # independent beams
    assert t0 == t1 == 15.0                           # the slowest rank's step time on both
    assert v0 == v1 == 2 * 64 * 1000.0 / 15.0         # all ranks' solves per second of that step


def test_single_rank_and_reference_arm_off_rank_zero():
    b = _bench()
    assert b._max_over_ranks(3.5, 1, "cpu") == 3.5
    assert b._job_rate(1, 1, 100.0) == 10.0

    class Args:
        workload = "beam_halo_1e5_depth6"
        steps = 1
        warmup = 3
    assert b.run_reference(Args(), 2, 1) is None      # rank 1: no work, nothing printed
