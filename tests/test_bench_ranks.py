"""The benchmark's multi-GPU host logic on two CPU processes (gloo): every
rank takes its own frames (weak scaling, no shared frame), the job's time is
the slowest rank's on every rank, and the whole-job rate counts all ranks'
frames."""
import json
import os
import socket
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_gloo():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, os.path.join(HERE, "ranks_worker.py")], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=300)
        assert p.returncode == 0, e[-2000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for r in outs:
        assert r["job_ms"] == 19.25                          # the slowest rank's time, on both ranks
        assert r["digests"][0] != r["digests"][1]            # distinct frames per rank
        assert abs(r["rate"] - 2 * 10 * 2 / 19.25e-3) < 1e-6
    assert outs[0]["digests"] == outs[1]["digests"]
