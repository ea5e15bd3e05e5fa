"""Every benchmark command in the committed ncu summaries (profiles/*.md)
still parses against bench.py's options (CPU): the summaries name commands
that run committed files only."""
import glob
import os
import re
import shlex
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bench_commands(path):
    text = open(path).read()
    cmds = []
    for block in re.findall(r"```\n(.*?)```", text, flags=re.S):
        block = block.replace("\\\n", " ")
        env = dict(re.findall(r'^([A-Z])="([^"]*)"', block, flags=re.M))
        for line in block.splitlines():
            if "bench.py" not in line:
                continue
            for part in line.split("bench.py")[1:]:
                part = re.split(r"&&|>|#|\|", part)[0]
                for k, v in env.items():
                    part = part.replace("$" + k, v)
                cmds.append(shlex.split(part))
    return cmds


SUMMARIES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))


@pytest.mark.parametrize("path", SUMMARIES, ids=[os.path.basename(p) for p in SUMMARIES])
def test_summary_commands_parse(path, monkeypatch):
    cmds = bench_commands(path)
    assert cmds, "no bench.py command in " + path
    for argv in cmds:
        monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
        args = bench.parse_args()
        assert args.impl == "mraid"
