"""One rank of the two-process check of the benchmark's multi-GPU host logic
(run by tests/test_bench_ranks.py with the gloo backend on CPU)."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402


def main():
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 19.25][rank]                 # each rank's own time
    job_ms = bench.max_over_ranks(ms)        # the job's time: the slowest rank
    det, mask, cal, fr = bench.setup_workload(2, rank)   # this rank's own frames
    digest = hashlib.sha256(fr.tobytes()).hexdigest()
    digests = [None] * world
    dist.all_gather_object(digests, digest)
    dist.barrier()
    print(json.dumps({"rank": rank, "job_ms": job_ms, "digests": digests,
                      "rate": bench.whole_job_rate(2, 10, world, job_ms)}), flush=True)
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
