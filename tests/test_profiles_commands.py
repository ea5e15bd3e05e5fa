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


def ncu_commands(path):
    text = open(path).read()
    out = []
    for block in re.findall(r"```\n(.*?)```", text, flags=re.S):
        block = block.replace("\\\n", " ")
        for line in block.splitlines():
            if line.strip().startswith("ncu ") or " ncu " in line:
                out.append(line[line.index("ncu "):])
    return out


@pytest.mark.parametrize("path", SUMMARIES, ids=[os.path.basename(p) for p in SUMMARIES])
def test_full_captures_name_one_kernel(path):
    """A capture that collects more than the launch-time metric covers one
    kernel (a -k regex without alternation) and at most three launches;
    every ncu command leaves the clocks alone."""
    for cmd in ncu_commands(path):
        assert "--clock-control none" in cmd, cmd
        launch_list = "--metrics gpu__time_duration.sum" in cmd and "--set" not in cmd
        if launch_list:
            continue
        m = (re.search(r'-k\s+"regex:([^"]+)"', cmd) or re.search(r'-k\s+regex:"([^"]+)"', cmd)
             or re.search(r"-k\s+regex:(\S+)", cmd))
        assert m, "a full capture must name its kernel: " + cmd
        assert "|" not in m.group(1), "one kernel per capture: " + cmd
        c = re.search(r"\s-c\s+(\d+)", cmd)
        assert c and int(c.group(1)) <= 3, "one to three launches per capture: " + cmd
