"""Host logic of bench.py: the lookup of a kernel's DRAM traffic in the ncu
summaries, which is used only while a summary's source hash matches the
current kernel sources, and scaled by arcs from a smaller workload of the
same family."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def write_profile(d, method, workload, arcs, h, nbytes):
    (d / f"{method}_{workload}.md").write_text(
        f"# {method}\n\n- workload = {workload} (n = 1; arcs = {arcs}; int32)\n"
        f"- kernel_source_hash = {h}   (sources)\n"
        f"- dram_bytes_per_launch = {nbytes}   (read + write)\n")


def test_traffic_found_only_for_the_current_sources(tmp_path):
    h = bench.kernel_source_hash("histocore")
    write_profile(tmp_path, "histocore", "rmat22", 1000, "0" * 16, 5000)
    b, src = bench.recorded_traffic("rmat22", "histocore", 1000, str(tmp_path))
    assert b is None and "no capture" in src
    write_profile(tmp_path, "histocore", "rmat22", 1000, h, 5000)
    b, src = bench.recorded_traffic("rmat22", "histocore", 1000, str(tmp_path))
    assert b == 5000 and "rmat22" in src


def test_traffic_scaled_by_arcs_within_a_family(tmp_path):
    h = bench.kernel_source_hash("peelone")
    write_profile(tmp_path, "peelone", "rmat22", 1000, h, 6000)
    b, src = bench.recorded_traffic("rmat24", "peelone", 4000, str(tmp_path))
    assert b == 24000 and "scaled" in src
    b, _ = bench.recorded_traffic("chunglu24", "peelone", 4000, str(tmp_path))
    assert b is None                      # another family is not scaled


def test_source_hash_covers_the_kernel_files():
    a, b = bench.kernel_source_hash("peelone"), bench.kernel_source_hash("histocore")
    assert len(a) == 16 and len(b) == 16 and a != b
