"""The committed ncu summaries that bench.py reads its `traffic` figure from:
one per bench workload, each with a 16-hex-digit kernel source hash and a
positive DRAM byte count per launch, within 15 % of the algorithmic bytes of
a full-size launch (a larger excess would mean re-reads or a wrong scaling)."""
import os
import re
import sys
import warnings

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

SITES = {"c4-batch64-fp32": None}  # batched: site count from the profile text


@pytest.mark.parametrize("workload", sorted(bench.WORKLOADS))
def test_profile_summary_parses(workload):
    path = os.path.join(ROOT, "profiles", f"step_kernel_{workload}.md")
    assert os.path.exists(path), path
    info = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            info[k.strip()] = v.strip().strip("`")
    assert re.fullmatch(r"[0-9a-f]{16}", info["kernel_source_hash"])
    traffic = float(info["dram_bytes_per_launch_full_size"])
    assert traffic > 0
    if info["kernel_source_hash"] != bench.kernel_hash():
        warnings.warn(f"{workload}: profile taken from another kernel source; bench reports traffic null")
    _, lattice, precision, n = bench.WORKLOADS[workload]
    m = re.search(r"algorithmic ([0-9.]+) B", open(path).read())
    per_site = float(m.group(1))
    sites = 24369565 if workload.startswith("c4") else n ** 3
    assert traffic <= 1.15 * per_site * sites
    assert traffic >= 0.95 * per_site * sites
