"""The multi-rank (replicas) host path of bench.py on CPU: two processes
joined over gloo (the backend bench.py takes when no GPU is present).

* max_over_ranks returns the slowest rank's time on every rank, and the
  barrier returns on both;
* under the reference arm only rank 0 works: another rank exits 0 at once,
  printing nothing.
"""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, sys
sys.path.insert(0, {root!r})
import bench
rank, world, local, pg = bench.dist_setup(2)
t = bench.max_over_ranks(pg, 1.5 + rank)      # rank 1 is the slower one
bench.barrier(pg)
print(json.dumps({{"rank": rank, "world": world, "local": local, "max": t}}), flush=True)
pg.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
    return env


def test_max_over_ranks_and_barrier_gloo():
    port = _free_port()
    code = RANK_SCRIPT.format(root=ROOT)
    procs = [subprocess.Popen([sys.executable, "-c", code], env=_env(r, 2, port), cwd=ROOT,
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    assert all(o["world"] == 2 and o["local"] == o["rank"] for o in outs)
    assert all(o["max"] == 2.5 for o in outs)


def test_reference_arm_other_ranks_exit_quietly():
    port = _free_port()
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0"], env=_env(1, 2, port), cwd=ROOT, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
