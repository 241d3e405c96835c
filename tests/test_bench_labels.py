"""The DRAM-traffic figures that bench.py reports next to its rooflines come
from ncu captures summarised under profiles/: each figure names its summary
and the commit whose kernel was captured.  These checks keep the labels
honest: the summary exists, names that commit and shows the figure."""
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _summary(path):
    full = os.path.join(ROOT, path)
    assert os.path.isfile(full), path
    with open(full, encoding="utf-8") as f:
        return f.read()


def _mb_figures(text):
    """Every number in the text (commas dropped), for matching a figure in MB."""
    return {float(x.replace(",", "")) for x in re.findall(r"\d[\d,]*\.\d+|\d[\d,]*", text)}


def test_headline_capture_label_matches_its_summary():
    assert bench.NCU_CAPTURES, "the headline roofline needs a capture"
    for kernel, cap in bench.NCU_CAPTURES.items():
        text = _summary(cap["summary"])
        assert cap["commit"] in text, (kernel, cap["commit"])
        mb = round(cap["dram_bytes"] / 1e6, 1)
        assert mb in _mb_figures(text), (kernel, mb)
        assert kernel not in bench.NCU_STALE


def test_secondary_capture_labels_match_their_summaries():
    for kernel, cap in bench.SECONDARY_CAPTURES.items():
        text = _summary(cap["summary"])
        assert cap["commit"] in text, (kernel, cap["commit"])
        assert f"`{kernel}" in text, kernel


def test_traffic_scales_with_the_particle_count():
    kernel, cap = next(iter(bench.NCU_CAPTURES.items()))
    same, note = bench.traffic_from_capture(kernel, cap["workload"], cap["n_particles"])
    assert same == cap["dram_bytes"] and cap["commit"] in note
    half, note2 = bench.traffic_from_capture(kernel, "another workload", cap["n_particles"] // 2)
    assert abs(half - cap["dram_bytes"] * (cap["n_particles"] // 2) / cap["n_particles"]) < 1.0
    assert "scaled by the particle count" in note2
    none, _ = bench.traffic_from_capture("no such kernel", cap["workload"], cap["n_particles"])
    assert none is None
