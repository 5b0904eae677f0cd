"""CPU: the commands quoted in profiles/ still run against today's bench.py -- every flag they
name (including the flags a note says to add) exists, and every ncu command leaves the clocks
alone (--clock-control none)."""
import glob
import os
import re
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))


def _commands(text):
    """Indented command blocks (backslash-continued lines joined)."""
    out, cur = [], ""
    for line in text.splitlines():
        if line.startswith("    ") and (cur or line.strip().startswith(("ncu", "python", "nvidia-smi"))):
            cur += " " + line.strip().rstrip("\\")
            if not line.rstrip().endswith("\\"):
                out.append(cur.strip())
                cur = ""
    return out


def _parse_bench(argv, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    return bench.parse_args()


def test_there_are_profiles():
    assert len(PROFILES) >= 4


@pytest.mark.parametrize("path", PROFILES, ids=os.path.basename)
def test_profile_commands_parse_and_keep_clocks(path, monkeypatch):
    text = open(path).read()
    cmds = [c for c in _commands(text) if "bench.py" in c]
    assert cmds, "no bench.py command"
    extra = []
    for m in re.finditer(r"add `([^`]*)`", text.replace("\n", " ")):
        extra += shlex.split(m.group(1))
    for c in cmds:
        if c.startswith("ncu"):
            assert "--clock-control none" in c
        argv = shlex.split(c.split("bench.py", 1)[1])
        _parse_bench(argv, monkeypatch)
        _parse_bench(argv + extra, monkeypatch)
