"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas only --
the hot path has no exchange step, so the only collectives are the barrier
and the max over ranks of the timed region)."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, ws: int, port: int, out_dir: str) -> None:
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_env() == (ws, rank, rank)
    local_ms = [12.0, 20.0][rank]
    total_ms, value = bench.job_throughput(local_ms, units_per_rank=1000, steps=5, ws=ws)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"total_ms": total_ms, "value": value}, f)


def _build_rank_main(rank: int, ws: int, port: int, out_dir: str, fail: bool) -> None:
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    calls = []

    def fake_build():
        calls.append(rank)
        if fail:
            raise RuntimeError("nvcc failed")

    ok = bench.build_once(ws, rank, fake_build)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"b{rank}.json"), "w") as f:
        json.dump({"ok": ok, "calls": calls}, f)


@pytest.mark.parametrize("fail", [False, True])
def test_build_handshake_reports_rank0_outcome_to_all(tmp_path, fail):
    port = _free_port()
    torch.multiprocessing.spawn(_build_rank_main, args=(2, port, str(tmp_path), fail), nprocs=2, join=True)
    d0, d1 = (json.load(open(tmp_path / f"b{r}.json")) for r in range(2))
    assert d0["calls"] == [0] and d1["calls"] == []  # only rank 0 builds
    assert d0["ok"] == d1["ok"] == (not fail)  # a failed build reaches every rank; nobody waits forever


def test_two_gloo_ranks_take_the_max_and_count_all_units(tmp_path):
    port = _free_port()
    torch.multiprocessing.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        d = json.load(open(tmp_path / f"r{r}.json"))
        assert d["total_ms"] == 20.0  # the slower rank's region
        assert d["value"] == pytest.approx(1000 * 5 * 2 / 0.020 / 1e6)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    total_ms, value = bench.job_throughput(8.0, units_per_rank=2000, steps=4, ws=1)
    assert total_ms == 8.0 and value == pytest.approx(2000 * 4 / 0.008 / 1e6)


def test_reference_arm_prints_only_on_rank_0():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert res.returncode == 0
    assert res.stdout.strip() == ""


def test_reference_arm_line_on_rank_0():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--ref-seconds", "1.5"], env=env, capture_output=True, text=True,
                         timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "Mqueries/s"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1 and d["higher_is_better"] is True
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["vs_baseline"] is None
    assert d["ms_per_step"] == pytest.approx(2073600 / (d["value"] * 1e6) * 1e3)
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "Mqueries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]

