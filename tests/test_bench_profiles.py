"""The bench's link to the committed ncu summaries (CPU only): every summary
it reads names a source hash and a DRAM figure that parse, and a summary whose
hash matches the current sources yields its traffic per launch or per unit."""
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_profile_summaries_parse():
    assert set(bench.PROFILE_OF_KERNEL) == set(bench.PROFILE_SOURCES)
    for kernel, name in bench.PROFILE_OF_KERNEL.items():
        path = os.path.join(ROOT, "profiles", name)
        assert os.path.exists(path), name
        text = open(path).read()
        m = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
        assert m, name
        figures = re.findall(r"dram_bytes_per_(launch|unit):\s*(\S+)", text)
        assert figures, name
        for _, v in figures:
            assert float(v) > 0, (name, v)
        if m.group(1) == bench.source_hash(kernel):
            t = bench.traffic_from_profile(kernel, 1.0e9)
            assert t is not None and t > 0, name


def test_source_hash_changes_with_sources():
    h = bench.source_hash("gram_tc_kernel")
    assert re.fullmatch(r"[0-9a-f]{64}", h)
    assert h != bench.source_hash("gram_tc_packed_kernel")


def test_kernels_without_a_summary_have_no_traffic():
    assert bench.traffic_from_profile("gram_f32_kernel") is None
    assert bench.traffic_from_profile("gram_f64_kernel") is None
