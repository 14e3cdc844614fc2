"""The committed ncu summaries the bench reads: every traffic entry names a
profile that exists and carries its command, and every source excerpt it is
keyed to is still found in the sources (so a kernel edit shows up as a digest
change, never as a silently missing excerpt)."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_entries_resolve():
    entries = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    assert entries
    for cls, e in entries.items():
        prof = open(os.path.join(ROOT, e["profile"])).read()
        assert "--clock-control none" in prof and "ncu " in prof, cls
        assert e["bytes_per_launch"] > 0, cls
        if "parts" in e:
            assert bench.parts_digest(e["parts"]) is not None, cls
        else:
            assert bench.kernel_digest(e["source"], e["kernel"]) is not None, cls


def test_every_profile_gives_its_command():
    d = os.path.join(ROOT, "profiles")
    for f in sorted(os.listdir(d)):
        if f.endswith(".md"):
            txt = open(os.path.join(d, f)).read()
            assert "```" in txt and "--clock-control none" in txt, f

