"""bench.py's host logic on CPU: the multi-rank reduction with two gloo ranks (each rank reports its
own step time, the job reports the maximum and counts every rank's replica: weak scaling, no
data-path collective), the oracle sample of the headline workload and the oracle timings of the
other workload shapes."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank
    m = bench.max_over_ranks(ms, dist, torch.device("cpu"))
    out[rank] = (m, bench.replica_throughput(1000, world, m))
    dist.destroy_process_group()


def test_two_rank_max_and_replica_throughput():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        m, v = out[r]
        assert m == 15.0
        assert v == pytest.approx(world * 1000 * 6 / 15e-3)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_throughput(10, 1, 1.0) == pytest.approx(60000.0)


def test_block_sample_ids():
    """The oracle's block sample: b^3 distinct ids forming the low-corner sub-box of the k^3 box."""
    import bench
    E = bench.block_elements(48, 8)
    assert E.size == 512 and np.unique(E).size == 512
    ex, ey, ez = E % 48, (E // 48) % 48, E // (48 * 48)
    assert ex.max() == ey.max() == ez.max() == 7 and min(ex.min(), ey.min(), ez.min()) == 0
    assert E[0] == 0 and E[1] == 1 and E[8] == 48 and E[64] == 48 * 48


def test_headline_workload_is_the_48cubed_p7_taylor_green():
    import bench
    W = bench.HEADLINE
    assert (W["k"], W["p"], W["warp"], W["Re"], W["Ma"], W["cfl"]) == (48, 7, 0.0, 1600.0, 0.1, 0.5)
    assert bench.nodes_of(W) == 56_623_104


def test_oracle_config_timings_cover_every_workload_shape():
    """The CPU-baseline leg times the oracle on every workload shape: the small Taylor-Green box (one
    residual and ten steps), the warped Taylor-Green sample, the warped vortex box and each p-sweep
    mesh's sample (no parity entries without a GPU)."""
    import bench
    t, parity = bench.oracle_config_timings()
    assert set(t) == {"tgv_4cubed_p3_affine", "tgv_16cubed_p4_warped", "vortex_8cubed_p4_warped"} | {
        f"tgv_psweep_p{p}_{k}cubed" for p, k in bench.PSWEEP_K.items()}
    for row in t.values():
        assert row["rhs_node_rhs_per_s"] > 0.0
    assert t["tgv_4cubed_p3_affine"]["dp5_10_steps_s"] > 0.0
    if not torch.cuda.is_available():
        assert parity == {}


def test_hbm_peak_reads_measured_file_or_falls_back():
    import bench
    v, src = bench.hbm_peak()
    assert v > 1000.0 and ("measured" in src or "fallback" in src)
