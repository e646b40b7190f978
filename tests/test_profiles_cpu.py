"""The ncu summaries under profiles/ name the commands that made them; those
commands must run committed files only (bench.py and its options), and the
traffic record bench.py reports must match the row kernel's current sources
or be absent."""
import json
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _tracked():
    r = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True)
    return set(r.stdout.split()) if r.returncode == 0 else None


def test_profile_commands_run_committed_files():
    tracked = _tracked()
    for name in os.listdir(PROFILES):
        if not name.endswith(".md"):
            continue
        text = open(os.path.join(PROFILES, name)).read()
        scripts = re.findall(r"python\s+([\w./-]+\.py)", text)
        assert scripts, f"{name} names no command"
        for sc in scripts:
            assert os.path.exists(os.path.join(ROOT, sc)), f"{name}: {sc} does not exist"
            assert not sc.startswith("_work"), f"{name}: {sc} is a working file"
            if tracked is not None:
                assert sc in tracked, f"{name}: {sc} is not committed"


def test_traffic_record_matches_sources():
    import bench
    rec = json.load(open(os.path.join(PROFILES, "traffic.json")))["k_rows2d"]
    assert rec["sources"] == list(bench.KERNEL_SOURCES["k_rows2d"])
    assert rec["dram_bytes_per_launch_full_size"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
    if rec["sources_sha256"] == bench.kernel_sources_sha256("k_rows2d"):
        assert bench.profile_traffic("k_rows2d") == rec["dram_bytes_per_launch_full_size"]
    else:
        assert bench.profile_traffic("k_rows2d") is None
