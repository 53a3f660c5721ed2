"""The committed profiler summaries and the sources they were taken from.

bench.py reports a kernel's DRAM traffic per launch (the roofline object's
`traffic`) only while the kernel's sources hash to the value stored with the
capture in profiles/traffic.json.  These checks keep that file honest: every
entry either matches its kernel's current sources or says why it does not,
and every summary gives the ncu commands that made it, each with the clock
control switched off (ncu otherwise locks the GPU clocks).
"""
import glob
import json
import os
import re

from paper_1908_03876_gb300.kernel_hash import KERNEL_SOURCES, kernel_source_hash

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _traffic():
    with open(os.path.join(PROFILES, "traffic.json")) as fh:
        return json.load(fh)


def test_traffic_entries_match_their_sources_or_say_why_not():
    tr = _traffic()
    entries = {k: v for k, v in tr.items() if isinstance(v, dict) and "sources_hash" in v}
    assert entries, "no kernel entries in traffic.json"
    for kernel, ent in entries.items():
        assert kernel in KERNEL_SOURCES, f"{kernel}: no source list in kernel_hash.KERNEL_SOURCES"
        if ent["sources_hash"] != kernel_source_hash(kernel):
            assert ent.get("note"), f"{kernel}: captured with other sources and no note says so"


def test_profile_summaries_give_their_commands():
    files = sorted(glob.glob(os.path.join(PROFILES, "*.md")))
    assert files
    for path in files:
        text = open(path, encoding="utf-8").read()
        runs = [ln for ln in text.splitlines() if re.match(r"\s*ncu\s+--", ln)]
        assert runs, f"{os.path.basename(path)}: no ncu command"
        for ln in runs:
            assert "--clock-control none" in ln, f"{os.path.basename(path)}: {ln.strip()}"
