"""The bench's multi-rank rules and its traffic record on CPU (no GPU).  The library is single-GPU:
under torchrun with WORLD_SIZE > 1 the native arm launches nothing (rank 0
prints one "unavailable" line, every rank exits 0, the library is never
loaded), and the reference arm (CPU only) runs on rank 0 alone."""
import json
import os
import re
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run_rank(rank, world, extra=()):
    env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
               MASTER_ADDR="127.0.0.1", MASTER_PORT="29511")
    # -X importtime lists every module the run imported (on stderr)
    return subprocess.run([sys.executable, "-X", "importtime", os.path.join(ROOT, "bench.py"),
                           *extra], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=300)


def test_native_arm_refuses_two_ranks_without_loading_the_library():
    for rank in (0, 1):
        r = _run_rank(rank, 2)
        assert r.returncode == 0, r.stderr[-2000:]
        # neither torch nor the library's binding was imported
        imported = re.findall(r"^import time:.*\|\s*([\w.]+)$", r.stderr, flags=re.M)
        assert "json" in imported                      # the listing itself works
        assert not any(m.split(".")[0] in ("torch", "paper_1306_4161_gb300")
                       for m in imported)
        lines = [l for l in r.stdout.splitlines() if l.strip()]
        if rank == 0:
            assert len(lines) == 1
            out = json.loads(lines[0])
            assert out["unavailable"] == bench.MULTI_GPU_UNAVAILABLE
            assert out["n_gpus"] == 2 and out["metric"] == bench.METRIC
        else:
            assert lines == []


def test_reference_arm_runs_on_rank_zero_only():
    # under torchrun every other rank leaves at once, without work or output
    import argparse
    args = argparse.Namespace(steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args, 1, 2) is None


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    # the bench reports the committed DRAM record only while the hash of the
    # kernel's file and the device headers it includes matches the capture's;
    # a changed source turns it into traffic_previous_capture
    import hashlib
    import json
    import shutil
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["bf16_pair_kernel"]
    assert rec["sources"] and all(os.path.exists(os.path.join(ROOT, f)) for f in rec["sources"])
    assert rec["dram_bytes_read"] > 0 and rec["dram_bytes_write"] > 0
    # a copy of the tree's files with the record's hash set to their current one
    for f in rec["sources"] + ["profiles/traffic.json"]:
        (tmp_path / os.path.dirname(f)).mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, f), tmp_path / f)
    h = hashlib.sha256()
    for f in rec["sources"]:
        h.update(open(tmp_path / f, "rb").read())
    data = json.load(open(tmp_path / "profiles" / "traffic.json"))
    data["bf16_pair_kernel"]["sha256_prefix"] = h.hexdigest()[:16]
    json.dump(data, open(tmp_path / "profiles" / "traffic.json", "w"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    total = rec["dram_bytes_read"] + rec["dram_bytes_write"]
    assert bench.traffic_record() == (total, True) and bench.measured_traffic() == total
    with open(tmp_path / rec["sources"][-1], "a") as fh:
        fh.write("\n")
    assert bench.traffic_record() == (total, False) and bench.measured_traffic() is None
