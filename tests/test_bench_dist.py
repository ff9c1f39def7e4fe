"""Host-side multi-rank logic of bench.py on CPU: two gloo ranks (replicas, weak
scaling) agree on the max of their step times and the sum of their keys, and the
reference arm under two ranks prints one line from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank: int, world: int, port: int) -> dict:
    env = dict(os.environ)
    env.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
    return env


_CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import bench
d = bench.Dist(2)
r = d.rank
d.barrier()
out = {"rank": r, "world": d.world, "max": d.max(1.5 + r), "sum": d.sum(10.0 * (r + 1))}
d.close()
print(json.dumps(out))
"""


def _run_ranks(argv_for_rank, world=2, timeout=300):
    port = _free_port()
    procs = [subprocess.Popen(argv_for_rank(r), env=_env(r, world, port), cwd=ROOT,
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for r in range(world)]
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            p.kill()
            o, e = p.communicate()
        outs.append((p.returncode, o, e))
    return outs


def test_two_gloo_ranks_reduce_max_and_sum():
    outs = _run_ranks(lambda r: [sys.executable, "-c", _CHILD, ROOT])
    for rc, o, e in outs:
        assert rc == 0, e
    lines = [json.loads(o.strip().splitlines()[-1]) for _, o, _ in outs]
    assert sorted(x["rank"] for x in lines) == [0, 1]
    for x in lines:
        assert x["world"] == 2
        assert x["max"] == 2.5        # max over ranks of the step time
        assert x["sum"] == 30.0       # whole-job units: the sum over ranks


def test_reference_arm_prints_once_under_two_ranks():
    argv = lambda r: [sys.executable, "bench.py", "--impl", "reference", "--gpus", "2",
                      "--steps", "2", "--warmup", "1", "--n", "20000"]
    outs = _run_ranks(argv)
    for rc, _, e in outs:
        assert rc == 0, e
    printed = [o.strip() for _, o, _ in outs if o.strip()]
    assert len(printed) == 1
    line = json.loads(printed[0].splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "keys/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_recorded_traffic_matches_sources_and_tuning(tmp_path, monkeypatch):
    """A recorded DRAM figure is returned only for the kernel sources it was captured on
    and, when its entry names a tuning, only under that tuning."""
    sys.path.insert(0, ROOT)
    import bench
    (tmp_path / "profiles").mkdir()
    entry = {"kernel": "k", "workload": "w", "source_hash": "h", "dram_bytes_per_launch": 7,
             "parts": {"tile_kernel<a>": 5, "small_kernel<b>": 2},
             "config": {"tile_shape": 3, "cutoff": 4096}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"entries": [entry]}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "device_source_hash", lambda: "h")
    assert bench.recorded_traffic("k", "w") == 7
    assert bench.recorded_traffic("k", "w", config={"tile_shape": 3, "cutoff": 4096}) == 7
    assert bench.recorded_traffic("k", "w", "small_kernel<", {"tile_shape": 3, "cutoff": 4096}) == 2
    assert bench.recorded_traffic("k", "w", config={"tile_shape": 3, "cutoff": 8192}) is None
    assert bench.recorded_traffic("k", "other") is None
    monkeypatch.setattr(bench, "device_source_hash", lambda: "changed")
    assert bench.recorded_traffic("k", "w") is None
