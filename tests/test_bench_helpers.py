"""Host helpers of the benchmark line: the DRAM traffic is taken from a profile summary only when that
summary was captured on the same kernel source and the same workload; the algorithmic bytes follow the
per-node and per-tetrahedron counts; one rank's whole-job rate is its own."""
import hashlib

import bench


def _summary(tmp_path, sha, tets, nodes, traffic="123.5e6"):
    p = tmp_path / "summary.md"
    p.write_text(f"# kernel\n\n- dram_bytes_per_launch_full_size: {traffic}\n- kernel_source_sha256: `{sha}`\n"
                 f"- workload_tets: {tets}\n- workload_nodes: {nodes}\n")
    return p


def test_traffic_needs_matching_kernel_source_and_workload(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("// kernel source\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    monkeypatch.setattr(bench, "KERNEL_SOURCE", str(src))
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(_summary(tmp_path, sha, 1000, 200)))
    assert bench.traffic_from_profile(1000, 200) == 123.5e6
    assert bench.traffic_from_profile(1000, 201) is None          # another mesh
    src.write_text("// kernel source, changed\n")
    assert bench.traffic_from_profile(1000, 200) is None          # the kernel changed since the capture
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(tmp_path / "missing.md"))
    assert bench.traffic_from_profile(1000, 200) is None


def test_algorithmic_bytes_of_the_element_pass():
    # 56 N bytes per node (3N + 4N + 3N + 4N FP32 values) and 80 bytes per tetrahedron
    assert bench.jvp_algorithmic_bytes(10, 0, 21) == 10 * 56 * 21
    assert bench.jvp_algorithmic_bytes(0, 7, 21) == 7 * 80


def test_single_rank_whole_job_rate():
    d = bench.Dist()                                               # not initialised: no process group
    rate, sec = bench.whole_job_rate(d, 600.0, 2.0)
    assert sec == 2.0 and rate == d.world * 300.0
