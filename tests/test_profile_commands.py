"""The commands recorded with the ncu summaries under profiles/ run committed
files only: every `python bench.py ...` in them parses with the bench's own
arguments, every summary gives at least one command, and every ncu command
leaves the GPU clocks alone."""
import glob
import os
import re
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUMMARIES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))


def _commands(text):
    out = []
    for block in re.findall(r"```\n(.*?)```", text, re.S):
        out += [c.strip() for c in block.replace("\\\n", " ").splitlines() if c.strip()]
    return out


@pytest.mark.parametrize("path", SUMMARIES, ids=[os.path.basename(p) for p in SUMMARIES])
def test_profile_commands_parse(path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    text = open(path).read()
    assert "_work" not in text
    cmds = _commands(text)
    if not cmds:   # a summary of another summary's capture names it
        assert re.search(r"`[a-z0-9_]+\.md`", text), path
        return
    for cmd in cmds:
        words = shlex.split(cmd)
        if "ncu" in words:
            assert "--clock-control" in words and words[words.index("--clock-control") + 1] == "none", cmd
        assert "bench.py" in words, cmd
        args = words[words.index("bench.py") + 1:]
        monkeypatch.setattr(sys, "argv", ["bench.py"] + args)
        bench.parse()   # exits (SystemExit) on an unknown flag
