"""Multi-process host logic of bench.py on CPU (gloo, world size 2): rank
discovery, barrier, max-over-ranks timing, per-rank sample batches, and the
reference arm printing only on rank 0; and that the full-size parity test
runs the launch shape bench.py times."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r'''
import os, sys, json
sys.path.insert(0, {root!r})
import bench
ws, rank, local = bench.dist_setup()
bench.barrier(ws)
t = bench.max_over_ranks(float(rank + 1) * 0.5, ws)
print(json.dumps({{"rank": rank, "ws": ws, "max": t, "seed": bench.SEED + 0x100000 * rank}}), flush=True)
import torch.distributed as dist
dist.destroy_process_group()
'''


def _launch(code, ws=2, port=29581):
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws),
               CUDA_VISIBLE_DEVICES="")
    procs = []
    for r in range(ws):
        e = dict(env, RANK=str(r), LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=e, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=240)
        assert p.returncode == 0, err
        outs.append(out)
    return outs


def test_two_ranks_barrier_and_max_over_ranks():
    outs = _launch(WORKER.format(root=ROOT))
    lines = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert sorted(l["rank"] for l in lines) == [0, 1]
    assert all(l["ws"] == 2 and l["max"] == 1.0 for l in lines)
    assert lines[0]["seed"] != lines[1]["seed"]  # each rank simulates its own sample batch


def test_reference_arm_prints_on_rank0_only():
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); sys.argv = ['bench.py', '--impl', 'reference', "
            f"'--steps', '1', '--warmup', '1']; import bench; bench.main()")
    outs = _launch(code, port=29582)
    printed = [o for o in outs if o.strip()]
    assert len(printed) == 1
    line = json.loads(printed[0].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    sys.path.insert(0, ROOT)
    import bench

    # the reference arm's line: the same metric and config as the GPU arm,
    # a cpu_baseline describing this run, and an e2e block with no copies
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT and line["higher_is_better"] is True
    assert line["config"]["workload"] == bench.WORKLOAD
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_full_size_parity_runs_the_benchmarked_shape():
    """The full-size GPU parity test checks the kernel and launch shape that
    bench.py times by default."""
    sys.path.insert(0, ROOT)
    import bench
    from tests.test_gpu_parity import BENCH_SHAPE

    assert tuple(bench.DEFAULT_VARIANT) == BENCH_SHAPE
