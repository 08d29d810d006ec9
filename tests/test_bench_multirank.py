"""The multi-GPU path of bench.py is replicas (one independent simulation per rank): the
job's time is the slowest rank's, its value all ranks' work over that time, and the
reference arm runs and prints on rank 0 only.  Checked with two gloo ranks on the CPU."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    import bench
    local_ms = [800.0, 1250.0][rank]
    total = bench.max_over_ranks(local_ms, world, "cpu")
    value = bench.job_value(world, 1000, 2000, total)
    buf = io.StringIO()
    args = bench.parse(["--impl", "reference", "--small", "--steps", "1", "--warmup", "0"])
    with redirect_stdout(buf):
        bench.reference_arm(args)
    dist.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"total": total, "value": value, "stdout": buf.getvalue()}, f)
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_rank0_reports(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(2)]
    assert r[0]["total"] == r[1]["total"] == 1250.0
    assert r[0]["value"] == r[1]["value"] == pytest.approx(2 * 1000 * 2000 / 1.25)
    assert r[1]["stdout"] == ""
    line = json.loads(r[0]["stdout"].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_value(1, 10, 20, 1000.0) == 200.0


def test_reference_line_keeps_the_contract():
    # the reference arm (the oracle, timed on the host) prints the CUDA arm's line: same
    # metric, unit, direction and scene, an e2e equal to its value with no copies
    sys.path.insert(0, ROOT)
    import bench
    args = bench.parse(["--impl", "reference", "--small", "--steps", "1", "--warmup", "0"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.reference_arm(args)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["higher_is_better"] is True
    assert line["unit"] == "particle-substeps/s" and line["value"] > 0
    # the same scene and metric as the CUDA arm; the workload says what the oracle ran
    sc = bench.workload(True)
    assert line["metric"] == bench.METRIC
    assert line["config"]["workload"].startswith(f"{sc.name}: {sc.n} fluid + {sc.nb} boundary")
    assert "one step = one regional substep" in line["config"]["workload"]
    assert "1 timed regional substeps" in line["cpu_baseline"]["sample"]
    assert line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle"
