"""Consistency of the committed documents with the tree: every file the
design notes and the README name exists, every profile summary names the
command that made it and runs only committed files, and the committed
traffic record points at kernel sources that exist."""
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SEARCH = ("", "tests", "profiles", "paper_1503_03635_gb300", os.path.join("paper_1503_03635_gb300", "csrc"),
          "oracle", "flsynth", "include")


def _exists(name):
    return any(os.path.exists(os.path.join(ROOT, d, name)) for d in SEARCH)


def test_files_named_in_the_documents_exist():
    missing = []
    for doc in ("DESIGN.md", "README.md"):
        with open(os.path.join(ROOT, doc)) as fh:
            text = fh.read()
        for name in set(re.findall(r"`([A-Za-z0-9_./-]+\.(?:py|md|cu|cuh|h|c|json|txt))`", text)):
            if name == "MEASURED_PEAKS.json":  # written by the measuring harness, not committed here
                continue
            if not _exists(name):
                missing.append((doc, name))
    assert not missing, missing


def test_profile_summaries_name_their_commands():
    prof = os.path.join(ROOT, "profiles")
    for name in sorted(os.listdir(prof)):
        path = os.path.join(prof, name)
        assert name.endswith((".md", ".txt", ".json")), name  # summaries only, nothing that runs
        assert os.path.getsize(path) < 64 * 1024, name
        if not name.endswith(".md"):
            continue
        with open(path) as fh:
            text = fh.read()
        assert re.search(r"^\s+(ncu |python )", text, re.M), f"{name} names no command"
        assert "_work" not in text, f"{name} refers to working files"


def test_traffic_record_points_at_existing_sources():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        d = json.load(fh)
    for kernel, per in d.items():
        for workload, e in per.items():
            src = os.path.join(ROOT, "paper_1503_03635_gb300", "csrc", e["source"])
            assert os.path.exists(src), (kernel, workload)
            assert e["dram_bytes_per_launch"] > 0
            assert re.fullmatch(r"[0-9a-f]{16}", e["source_sha256_16"])
