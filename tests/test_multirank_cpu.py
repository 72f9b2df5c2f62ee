"""The benchmark's multi-rank host logic on CPU with two gloo ranks: max-over-ranks timing and the
whole-job value (one independent replica per rank, no collective on the data path)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local = [100.0 + 50.0 * rank, 10.0 * (ws - rank), 7.0]
    got = bench.max_over_ranks(local, ws, device="cpu")
    value = bench.whole_job_tflops(1e12, ws, got[0])
    out[rank] = (got, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_and_whole_job_value():
    ws, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as mgr:  # no fork of this multi-threaded process
        out = mgr.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        got, value = res[rank]
        assert got == [150.0, 20.0, 7.0]           # element-wise max over the ranks
        assert value == pytest.approx(1e12 * ws / 0.150 / 1e12)  # both replicas in the slowest rank's time


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1, device="cpu") == [3.0, 4.0]
    assert bench.whole_job_tflops(2e12, 1, 1000.0) == pytest.approx(2.0)


def test_host_lapack_point():
    """The bench's secondary host point (numpy's LAPACK Cholesky of the same K) reports a positive
    rate, or says why it could not run."""
    import bench
    r = bench.cpu_library_cholesky(256, 8)
    assert r["kind"].startswith("numpy.linalg.cholesky")
    assert "unavailable" in r or (r["n"] == 256 and r["s"] > 0 and r["tflops"] > 0 and r["cores"] >= 1)
