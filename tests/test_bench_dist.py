"""Host-side logic of bench.py on CPU: two gloo ranks (replicas, weak scaling) agree on
the max of their step times and the sum of their keys, and the reference arm under two
ranks prints one line from rank 0 only; recorded DRAM traffic applies only to the kernel
sources and tuning it was captured under; the sort roofline's arithmetic."""
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
    monkeypatch.setattr(bench, "device_source_hash", lambda *a: "h")
    assert bench.recorded_traffic("k", "w") == 7
    assert bench.recorded_traffic("k", "w", config={"tile_shape": 3, "cutoff": 4096}) == 7
    assert bench.recorded_traffic("k", "w", "small_kernel<", {"tile_shape": 3, "cutoff": 4096}) == 2
    assert bench.recorded_traffic("k", "w", config={"tile_shape": 3, "cutoff": 8192}) is None
    assert bench.recorded_traffic("k", "other") is None
    monkeypatch.setattr(bench, "device_source_hash", lambda *a: "changed")
    assert bench.recorded_traffic("k", "w") is None


def test_sort_roofline_arithmetic(monkeypatch):
    """The sort roofline: the dominant kernel is the phase with the longer mean time; its
    achieved rate is 2 * 4 B per key it moves over that time, and the fraction divides by
    the given peak; the other phase and the whole call are reported beside it."""
    sys.path.insert(0, ROOT)
    import bench
    import paper_1107_3622_gb300 as ks
    ks.load()
    monkeypatch.setattr(bench, "recorded_traffic", lambda *a, **k: None)
    stats = {"large_keys": 100_000_000, "small_keys": 7_000_000}
    phases = [[0.01, 0.40, 0.25], [0.01, 0.42, 0.25], [0.02]]  # a short record is skipped
    r = bench.sort_roofline(ks, stats, phases, 0.70, 7_000_000, 6000.0, "measured")
    assert r["launch_ms"] == 0.41 and r["algorithmic_bytes_per_launch"] == 800_000_000
    assert r["achieved"] == round(800e6 / 0.41e-3 / 1e9, 1)
    assert r["frac"] == round(800e6 / 0.41e-3 / 1e9 / 6000.0, 4)
    assert r["finisher"]["algorithmic_bytes_per_launch"] == 56_000_000
    assert r["finisher"]["launch_ms"] == 0.25
    assert r["whole_call"]["algorithmic_bytes_per_call"] == 856_000_000
    assert r["whole_call"]["frac"] == round(856e6 / 0.70e-3 / 1e9 / 6000.0, 4)
    assert r["timing"].startswith("library phase events") and "2 timed steps" in r["timing"]
    # a finisher that takes longer becomes the dominant kernel
    r2 = bench.sort_roofline(ks, stats, [[0.01, 0.1, 0.3]], 0.45, 7_000_000, 6000.0, "measured")
    assert r2["kernel"].startswith("small_kernel") and "partition_passes" in r2


def test_recorded_traffic_checks_the_files_an_entry_names(tmp_path, monkeypatch):
    """An entry that names its source files is checked against the hash of those files
    alone, so a change elsewhere in the device sources leaves it valid."""
    sys.path.insert(0, ROOT)
    import bench
    (tmp_path / "profiles").mkdir()
    entries = [{"kernel": "k", "workload": "w", "sources": ["a.cuh"], "source_hash": "ha",
                "dram_bytes_per_launch": 3},
               {"kernel": "k2", "workload": "w", "source_hash": "ha", "dram_bytes_per_launch": 4}]
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"entries": entries}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "device_source_hash",
                        lambda files=bench.DEVICE_SOURCES: "ha" if tuple(files) == ("a.cuh",) else "all")
    assert bench.recorded_traffic("k", "w") == 3
    assert bench.recorded_traffic("k2", "w") is None
