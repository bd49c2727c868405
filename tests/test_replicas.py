"""bench.py with N > 1: every rank runs an independent replica (the method is not sharded here),
the timed region ends with the slowest rank, and the whole-job value counts every replica's
iterations.  Checked with two gloo ranks on the CPU, launched the way the multi-GPU bench is."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_replicas_report_the_slowest_rank_and_the_whole_job(tmp_path):
    pytest.importorskip("torch.distributed")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "tests", "replica_worker.py")]
    env = dict(os.environ, OMP_NUM_THREADS="1", REPLICA_OUT=str(tmp_path))
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=240)
    assert out.returncode == 0, out.stderr[-2000:]
    rows = [json.loads((tmp_path / f"rank{r}.json").read_text()) for r in range(2)]
    assert sorted(r["rank"] for r in rows) == [0, 1]
    for r in rows:
        assert r["world"] == 2
        assert r["t"] == 1.5                       # the slower replica's time, on every rank
        assert r["value"] == pytest.approx(2 * 10 / 1.5)
