"""The DRAM traffic that bench.py reports comes from a committed ncu capture
(profiles/<kernel>.json beside its summary profiles/<kernel>.md) only while
the kernel's sources are those the capture ran: the JSON records a hash of
them, and a changed source makes the traffic null.  The summaries give the
full command that produced them, and every ncu command leaves the GPU's
clocks alone (--clock-control none)."""
import glob
import hashlib
import json
import os
import re

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _tree(tmp_path, kernel_src: bytes, record: dict):
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_2406_12202_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_bytes(kernel_src)
    (tmp_path / "profiles" / "k_test.json").write_text(json.dumps(record))


def test_traffic_follows_the_recorded_source_hash(tmp_path, monkeypatch):
    src = b"__global__ void k() {}\n"
    _tree(tmp_path, src, {"source_sha16": hashlib.sha256(src).hexdigest()[:16],
                          "traffic_bytes_per_launch": 123456.0})
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("k_test", ("k.cu",)) == 123456.0
    # any change to the source (a comment too) makes the capture stale
    (tmp_path / "paper_2406_12202_gb300" / "csrc" / "k.cu").write_bytes(src + b"// edit\n")
    assert bench.profiled_traffic("k_test", ("k.cu",)) is None
    # a missing capture, or one without a traffic figure, reports none
    assert bench.profiled_traffic("k_absent", ("k.cu",)) is None


def test_traffic_null_when_the_capture_has_no_figure(tmp_path, monkeypatch):
    src = b"x"
    _tree(tmp_path, src, {"source_sha16": hashlib.sha256(src).hexdigest()[:16],
                          "traffic_bytes_per_launch": None})
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("k_test", ("k.cu",)) is None


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(PROFILES, "*.json"))),
                         ids=os.path.basename)
def test_committed_captures_are_well_formed(path):
    with open(path) as f:
        rec = json.load(f)
    assert re.fullmatch(r"[0-9a-f]{16}", rec["source_sha16"])
    t = rec["traffic_bytes_per_launch"]
    assert t is None or t > 0
    # the summary it belongs to
    assert os.path.exists(path[:-5] + ".md")


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(PROFILES, "*.md"))),
                         ids=os.path.basename)
def test_summaries_give_their_command_and_keep_clocks(path):
    with open(path) as f:
        text = f.read()
    cmds = [ln for ln in text.splitlines() if re.search(r"\bncu\b", ln) and "--" in ln]
    assert cmds, "a summary names the ncu command that produced it"
    for ln in cmds:
        assert "--clock-control none" in ln, ln
