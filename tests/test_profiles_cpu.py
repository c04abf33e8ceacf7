"""The ncu summaries under profiles/ name the commands that made them; those
commands must still be valid invocations of the committed bench.py (every
flag known, the warm-up at least 3), so that anyone can rerun them."""
import glob
import os
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _bench_commands():
    out = []
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            line = line.strip()
            if line.startswith("python bench.py"):
                out.append((os.path.basename(path), line))
    return out


CMDS = _bench_commands()


def test_every_summary_names_a_bench_command():
    names = {os.path.basename(p) for p in glob.glob(os.path.join(ROOT, "profiles", "*.md"))}
    assert names and names <= {n for n, _ in CMDS}


@pytest.mark.parametrize("name,cmd", CMDS)
def test_summary_command_parses(name, cmd):
    argv = shlex.split(cmd)[2:]
    # per-format captures write the format as a placeholder letter
    argv = ["fp32" if a == "F" else a for a in argv]
    args = bench.make_parser().parse_args(argv)
    assert args.warmup >= 3, (name, cmd)
    for fmt in args.obstacle_formats.split(","):
        assert fmt in bench.FORMAT_KEYS, (name, fmt)
