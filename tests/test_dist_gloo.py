"""The multi-GPU path is replicas only: N ranks each run the whole workload,
synchronise with a barrier and report the slowest rank's time.  Two gloo ranks
on the CPU check that rendezvous, barrier and the max-over-ranks throughput
of bench.py agree across ranks."""
import json
import os
import socket
import subprocess
import sys
import textwrap

REPO = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))

SCRIPT = textwrap.dedent("""
    import json, sys
    sys.path.insert(0, %r)
    import bench
    ws, rank, local = bench.dist()
    bench.barrier(ws)
    value, ms = bench.replica_value(1000, ws, 10.0 + 5.0 * rank)   # rank 1 is slower
    print(json.dumps({"rank": rank, "ws": ws, "local": local, "value": value, "ms": ms}))
""") % REPO


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_replicas_report_the_slowest_rank():
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", SCRIPT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["ws"] == 2
        assert o["ms"] == 15.0                       # max over ranks
        assert abs(o["value"] - 2 * 1000 / 15e-3) < 1e-6
    assert sorted(o["rank"] for o in outs) == [0, 1]


def test_single_process_needs_no_process_group():
    import bench
    value, ms = bench.replica_value(1000, 1, 20.0)
    assert ms == 20.0 and abs(value - 1000 / 20e-3) < 1e-9
