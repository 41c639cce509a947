"""The multi-rank path of bench.py on the CPU (gloo, world size 2): the
runs are independent replicas, so the ranks exchange only the timing
reductions (the maximum of the ranks' times, the sum of their cell
updates) and barriers; the reference arm runs on rank 0 alone and the
other ranks exit without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(code, world=2, timeout=120):
    port = _port()
    procs = []
    for r in range(world):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r),
                   WORLD_SIZE=str(world), LOCAL_RANK=str(r), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", code], cwd=ROOT, env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=timeout)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_timing_reductions_over_two_gloo_ranks():
    code = ("import bench, json, torch.distributed as dist\n"
            "r, w, l = bench.dist_setup()\n"
            "assert dist.get_backend() == 'gloo' and w == 2\n"
            "mx = bench.reduce_max(1.5 + r, w)\n"
            "sm = bench.reduce_sum(10.0 * (r + 1), w)\n"
            "bench.barrier(w)\n"
            "print(json.dumps([r, mx, sm]))\n"
            "dist.destroy_process_group()\n")
    outs = _run(code)
    got = sorted(json.loads(o.strip().splitlines()[-1]) for o in outs)
    assert got == [[0, 2.5, 30.0], [1, 2.5, 30.0]]


def test_reference_arm_prints_on_rank_zero_only():
    pytest.importorskip("numpy")
    code = ("import sys, bench\n"
            "sys.argv = ['bench.py', '--impl', 'reference', '--gpus', '2', '--steps', '1', '--warmup', '1',"
            " '--n', '16']\n"
            "bench.main()\n")
    outs = _run(code, timeout=300)
    lines = [o.strip().splitlines() for o in outs]
    assert len(lines[1]) == 0 or not any(l.startswith("{") for l in lines[1])
    line = json.loads(lines[0][-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
