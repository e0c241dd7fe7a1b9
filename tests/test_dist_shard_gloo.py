"""Host side of the row-sharded group on CPU (no GPU): two gloo processes check the
allreduce adapter that ``Problem.set_comm`` takes (sum and max, float32 and float64) and the
contiguous row partition."""
import os
import socket
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def run_group(tmp_path, world, extra=()):
    port = free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen(
            [sys.executable, os.path.join(ROOT, "tests", "shard_worker.py"), "--mode", "cpu",
             "--out", str(tmp_path / f"r{r}.npz"), *extra], env=env, cwd=ROOT,
            stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    for pr in procs:
        out, err = pr.communicate(timeout=240)
        assert pr.returncode == 0, err[-2000:]
    return [np.load(tmp_path / f"r{r}.npz") for r in range(world)]


def test_allreduce_adapter_and_row_partition(tmp_path):
    res = run_group(tmp_path, 2, ("--n", "1001"))
    want = np.arange(4) * 2 + 10.0
    for r in res:
        np.testing.assert_array_equal(r["sum"], want)
        np.testing.assert_array_equal(r["max"], np.array([1.0, 0.0], np.float32))
    (a0, b0), (a1, b1) = res[0]["rows"], res[1]["rows"]
    assert (a0, b0, a1, b1) == (0, 501, 501, 1001)


def test_row_partition_covers_the_pool():
    sys.path.insert(0, ROOT)
    from paper_2409_07392_gb300.api import shard_rows
    for n in (1, 7, 1000, 1_000_003):
        for world in (1, 2, 3, 8):
            spans = [shard_rows(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
