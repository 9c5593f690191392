"""The benchmark's link to the committed ncu summaries: a summary's DRAM counters are used
only while the kernel sources it was taken on are unchanged (per-section digests), and the
algorithmic bytes the summaries and the roofline divide by follow the per-unit model on the
workloads' trees."""
from __future__ import annotations

import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

SRC = """// ------------------------------------------------------------------ first
int a;
// ------------------------------------------------------------------ stream schedule
int b;
int c;
// ------------------------------------------------------------------ wide schedule
int d;
"""


def test_without_sections_drops_a_section_up_to_the_next_header():
    out = bench.without_sections(SRC, {"stream schedule"})
    assert "int b;" not in out and "int c;" not in out
    assert "int a;" in out and "int d;" in out and "wide schedule" in out
    assert bench.without_sections(SRC, set()) == SRC
    both = bench.without_sections(SRC, {"stream schedule", "wide schedule"})
    assert both.splitlines() == SRC.splitlines()[:2]


def test_kernel_sources_have_the_sections_the_summaries_name():
    text = open(os.path.join(ROOT, "paper_2605_19928_gb300", "csrc", "kernels.cu")).read()
    headers = set(re.findall(r"^// -{10,} (.+)$", text, flags=re.M))
    for name in os.listdir(os.path.join(ROOT, "profiles")):
        summary = open(os.path.join(ROOT, "profiles", name)).read()
        x = re.search(r"kernels_digest_excludes:\s*(.+)", summary)
        if x:
            for section in x.group(1).split(","):
                assert section.strip() in headers, (name, section)
    # leaving a section out changes the digest, and only then
    assert bench.kernels_digest(("stream schedule",)) != bench.kernels_digest()
    assert bench.kernels_digest(("no such section",)) == bench.kernels_digest()


def test_profiled_traffic_needs_a_matching_digest(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    good = bench.kernels_digest(("stream schedule",))
    (prof / "update_toy.md").write_text(f"kernels_digest: {good}\nkernels_digest_excludes: stream schedule\n"
                                        "dram_bytes_per_launch: 1234\n")
    (prof / "update_stale.md").write_text("kernels_digest: 0000000000000000\ndram_bytes_per_launch: 99\n")
    (prof / "update_full.md").write_text(f"kernels_digest: {good}\ndram_bytes_per_launch: 5\n")
    real_root = bench.ROOT
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "paper_2605_19928_gb300").symlink_to(os.path.join(real_root, "paper_2605_19928_gb300"))
    assert bench.profiled_traffic("update", "toy") == 1234.0
    assert bench.profiled_traffic("update", "stale") is None
    assert bench.profiled_traffic("update", "full") is None  # a full-source digest would differ
    assert bench.profiled_traffic("update", "missing") is None


def _oracle_shape(om, spec):
    """The bench's tree shape (nodes, hands, regret rows per player, terminals), taken from
    the oracle's own tree."""
    o = om.Oracle(spec, variant="dcfr", threads=1)
    rows, ends = [0, 0], 0
    for nd in o.nodes():
        if nd["type"] == 0:
            rows[nd["player"]] += nd["n_actions"]
        elif nd["type"] in (1, 2, 4):
            ends += 1
    return {"nodes": o.n_nodes, "hands": o.n_hands, "rows": rows, "terminals": ends}


def _profile_figure(name, pattern):
    text = open(os.path.join(ROOT, "profiles", name)).read()
    return int(re.search(pattern, text).group(1).replace(",", ""))


def test_roofline_numerators_of_the_summaries(oracle_mod):
    """The algorithmic bytes the committed summaries divide by: the benchmark's per-unit
    model applied to the workloads' trees, built here by the oracle."""
    from paper_2605_19928_gb300 import synth
    river = _oracle_shape(oracle_mod, bench.workload_spec(0))
    assert river["hands"] == 1081
    # the resident launch: 20 iterations of both players' update and terminal launches
    want = _profile_figure("resident_river1081.md", r"algorithmic bytes per launch \| .*= ([\d,]+) B")
    per_iter = 2 * (bench.algorithmic_bytes(river, "update", 4) + bench.algorithmic_bytes(river, "terminal", 4))
    assert 20 * per_iter == want
    batch = [_oracle_shape(oracle_mod, s) for s in synth.batch_rivers(256)]
    total = sum(bench.algorithmic_bytes(sh, "update", 4) for sh in batch)
    half = sum(bench.algorithmic_bytes(sh, "update", 4) for sh in batch[:128])
    text = open(os.path.join(ROOT, "profiles", "update_batch256.md")).read()
    assert f"{int(half):,}" in text and f"{int(total):,}" in text
