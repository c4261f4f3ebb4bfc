"""The N > 1 host path of bench.py on CPU: two gloo ranks (processes started
with spawn, rendezvous on 127.0.0.1).  The path shards only as replicas, so
the one exchange is the timing reduction: the job's step time is the slowest
rank's, and the rate counts every rank's points.  The reference arm runs on
rank 0 only; the others exit 0 without work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        # rank r took (r + 1) ms for a step of 1000 points
        ms, rate = bench.whole_job_rate(1.0 + rank, 1000, ws)
        out[rank] = (ms, rate, bench._dist())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_reduction():
    ws, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(ws, port, out), nprocs=ws, join=True, start_method="spawn")
        res = dict(out)
    for rank in range(ws):
        ms, rate, (w, r, local) = res[rank]
        assert (w, r, local) == (ws, rank, rank)
        assert ms == 2.0                      # the slowest rank's time, on every rank
        assert rate == pytest.approx(2 * 1000 / 2e-3)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class Args:
        steps, warmup, gpus = 1, 0, 2

    # rank 1 returns before loading the oracle or printing anything
    assert bench.reference_main(Args()) == 0


def test_single_rank_rate():
    import bench
    ms, rate = bench.whole_job_rate(0.5, 2000, 1)
    assert ms == 0.5 and rate == pytest.approx(2000 / 0.5e-3)


def test_bench_series_depth_is_the_truncation_study_default():
    """The benchmark's Gimenez depth is the one the truncation study picks
    (tests/golden/gimenez_truncation.json): the smallest within 1e-5 over the
    long-cadence priors."""
    import json
    import bench
    g = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "gimenez_truncation.json")))
    assert bench.N_J == g["default_n_j"]
