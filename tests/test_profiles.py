"""The ncu summaries under profiles/ (CPU): each is short text, names the
command that produced it, every ncu command leaves the clocks alone
(--clock-control none), and every bench.py command line in them is still
accepted by bench.py's own argument parser (the autotuner's by its own)."""
import os
import re
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")
FILES = sorted(f for f in os.listdir(PROFILES))


def _joined(text):
    return re.sub(r"\\\n\s*", " ", text)   # shell continuation lines


@pytest.mark.parametrize("name", FILES)
def test_summary_is_short_text_with_its_command(name):
    path = os.path.join(PROFILES, name)
    assert name.endswith((".md", ".txt"))
    assert os.path.getsize(path) < 16 * 1024
    text = _joined(open(path).read())
    assert "python bench.py" in text or "python -m paper_1908_09606_gb300" in text
    for line in text.splitlines():
        if line.lstrip().startswith(("#", "|")):
            continue   # headings and table rows describe a capture, they do not run one
        if re.search(r"\bncu\s+--", line):
            assert "--clock-control none" in line, (name, line)


@pytest.mark.parametrize("name", FILES)
def test_bench_command_lines_parse(name, monkeypatch):
    import bench
    text = _joined(open(os.path.join(PROFILES, name)).read())
    cmds = re.findall(r"python bench\.py([^\"`\n|>$]*)", text)
    for args in cmds:
        monkeypatch.setattr(sys, "argv", ["bench.py"] + shlex.split(args))
        bench.parse()   # raises SystemExit on an option bench.py no longer has


@pytest.mark.parametrize("name", FILES)
def test_autotune_command_lines_parse(name):
    from paper_1908_09606_gb300 import autotune
    text = _joined(open(os.path.join(PROFILES, name)).read())
    for args in re.findall(r"python -m paper_1908_09606_gb300\.autotune([^\"`\n|>$]*)", text):
        autotune.parser().parse_args(shlex.split(args))
