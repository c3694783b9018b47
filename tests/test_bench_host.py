"""Host-side logic of bench.py, on the CPU: the whole-job figures of a multi-rank run
(world_size 2 over gloo) and the reference arm (the FP64 oracle timed on the host cores)."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t, e2e = bench.combine_ranks(10.0 * (rank + 1), 100.0 * (rank + 1), world, "cpu")
    out.put((rank, t, e2e, bench.job_mlups(1000, 10, world, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_two_processes_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, e2e, mlups in res:
        assert t == 20.0            # slowest rank's time
        assert e2e == 200.0         # world x slowest rank's end-to-end rate
        assert mlups == pytest.approx(2 * 1000 * 10 / 0.020 / 1e6)


def test_combine_ranks_single_rank_is_identity():
    import bench

    assert bench.combine_ranks(3.0, 7.0, 1, "cpu") == (3.0, 7.0)


def test_reference_arm_prints_one_json_line():
    env = dict(os.environ)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3",
                        "--warmup", "1", "--cpu-seconds", "0.3", "--dims", "32", "32", "32"], capture_output=True, text=True, env=env,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "32x32x32" in d["cpu_baseline"]["sample"] and "sub-lattice" not in d["cpu_baseline"]["sample"]
    assert d["cpu_baseline"]["single_core"]["cores"] == 1


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"], capture_output=True,
                       text=True, env=env, timeout=120, cwd=ROOT)
    assert r.returncode == 0 and r.stdout.strip() == ""
