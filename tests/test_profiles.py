"""The committed ncu summaries stay usable: bench.py reports roofline.traffic from the hop
summary only while its kernel-source hash matches the current sources, and every bench.py
command the summaries record must still parse with today's flags (no GPU)."""

import os
import re
import shlex
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

PROFILES = os.path.join(ROOT, "profiles")


def test_hop_summary_matches_the_kernel_sources():
    """A change to fs_hop.cuh, fs_common.cuh or fs_launch.cuh needs a new DRAM capture of the hop
    kernels (profiles/hop_kernel_16x32.md); until then the bench reports no traffic."""
    ratio = bench.hop_traffic_ratio("16x32")
    assert ratio is not None
    assert 0.9 < ratio < 1.3


def _bench_commands(text):
    """bench.py argument lists of the commands in a summary's code blocks (continuations joined)."""
    out = []
    for block in re.findall(r"```\n(.*?)```", text, flags=re.S):
        cmd = block.replace("\\\n", " ")
        for line in cmd.splitlines():
            words = shlex.split(line)
            if "bench.py" in words:
                out.append(words[words.index("bench.py") + 1:])
    return out


def test_recorded_bench_commands_parse():
    n = 0
    for name in sorted(os.listdir(PROFILES)):
        if not name.endswith(".md"):
            continue
        with open(os.path.join(PROFILES, name)) as f:
            for argv in _bench_commands(f.read()):
                bench.build_parser().parse_args(argv)
                n += 1
    assert n >= 3
