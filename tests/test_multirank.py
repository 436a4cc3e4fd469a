"""The multi-rank path of the benchmark on CPU (gloo, world size 2): every
rank measures its own seeded copy of the workload (weak scaling, replicas,
no data-path collective), and the whole-job figures are the slowest rank's
time and the work of all ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import workloads as W
        ms, units = bench.whole_job([3.0, 5.0][rank], [100, 250][rank], dist, "cpu")
        seed = bench.rank_seed(2024, rank)
        fb = W.fit_batch(seed, 2, 20, dtype=np.float32)
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), ms=ms, units=units, seed=seed,
                 y=fb.y, x=fb.x)
    finally:
        dist.destroy_process_group()


def test_two_ranks_whole_job_and_distinct_replicas(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = [np.load(tmp_path / f"r{i}.npz") for i in range(2)]
    for ri in r:
        assert float(ri["ms"]) == 5.0 and float(ri["units"]) == 350.0
    assert int(r[0]["seed"]) != int(r[1]["seed"])
    # each rank draws its own replica of the workload
    assert not np.array_equal(r[0]["y"], r[1]["y"])


def test_single_rank_whole_job_is_local():
    import bench
    assert bench.whole_job(2.5, 64, None) == (2.5, 64.0)


def test_reference_arm_prints_its_line():
    """bench.py --impl reference times the oracle on the host and prints the
    contract's line (runs on CPU)."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True,
                         timeout=600, check=True).stdout
    line = json.loads(out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "queries/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["higher_is_better"] is True and line["steps"] == 2
