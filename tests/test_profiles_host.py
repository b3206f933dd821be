"""Every ncu summary under profiles/ names the command that produced it; the bench
invocations in those commands must still be accepted by bench.py's argument parser."""
import glob
import importlib.util
import os
import re
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUMMARIES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))


def _bench_commands(path):
    text = open(path).read().replace("\\\n", " ")  # join continued lines
    cmds = []
    for line in text.splitlines():
        for m in re.finditer(r"python bench\.py([^|&>`]*)", line):
            cmds.append(shlex.split(m.group(1)))
    return cmds


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_for_profiles", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_every_summary_names_its_command():
    assert SUMMARIES
    for p in SUMMARIES:
        text = open(p).read()
        assert "python bench.py" in text or "ncu " in text, p


@pytest.mark.parametrize("path", SUMMARIES, ids=[os.path.basename(p) for p in SUMMARIES])
def test_bench_commands_in_summaries_parse(path, bench, monkeypatch):
    for args in _bench_commands(path):
        monkeypatch.setattr(sys, "argv", ["bench.py"] + args)
        bench.parse()  # exits (SystemExit) on an unknown option or value
