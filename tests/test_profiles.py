"""The committed ncu summaries: short text with the command that made them, every ncu run with
--clock-control none, nothing that points at working files, and every traffic figure the
bench reads present."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")
FILES = sorted(f for f in os.listdir(PROFILES))


def _commands(text):
    """The ncu invocations of a summary's code blocks, continuation lines joined."""
    blocks = re.findall(r"```(.*?)```", text, flags=re.S)
    cmds = []
    for b in blocks:
        joined = re.sub(r"\\\n\s*", " ", b)
        cmds += [ln.strip() for ln in joined.splitlines() if ln.strip().startswith("ncu ")]
    return cmds


@pytest.mark.parametrize("name", FILES)
def test_summary_is_short_text_with_its_command(name):
    assert name.endswith((".md", ".txt")), name
    path = os.path.join(PROFILES, name)
    assert os.path.getsize(path) < 16 * 1024, name
    text = open(path).read()
    assert "```" in text, "%s quotes no command" % name
    for cmd in _commands(text):
        assert "--clock-control none" in cmd, (name, cmd)
    for word in ("_work/", "gpurun", "/root/"):
        assert word not in text, (name, word)


def test_every_traffic_figure_the_bench_reads_exists():
    import bench
    src = open(os.path.join(ROOT, "bench.py")).read()
    tags = set(re.findall(r'"((?:cg|mg)_[a-z0-9_]+_64cube(?:#[a-z]+)?)"', src))
    assert tags
    for tag in sorted(tags):
        assert bench.traffic_per_dof(tag) is not None, tag
