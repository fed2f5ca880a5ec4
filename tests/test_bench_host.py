"""Host-side pieces of the benchmark without a GPU: the traffic record is keyed
to the kernel sources without their comments (a documentation change keeps it,
a code change drops it), and the flop counts behind the roofline."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_kernel_source_hash_ignores_comments_only(tmp_path, monkeypatch):
    a = tmp_path / "a.cuh"
    a.write_text("int f(int x) {\n  return x + 1;  // one more\n}\n/* note */\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC_SOURCES", ("a.cuh",))
    h0 = bench.kernel_sources_sha256()
    a.write_text("// header\nint f(int x) {\n  return x + 1;  // one more, reworded\n}\n\n/* another\n note */\n")
    assert bench.kernel_sources_sha256() == h0
    a.write_text("int f(int x) {\n  return x + 2;\n}\n")
    assert bench.kernel_sources_sha256() != h0


def test_per_scp_iteration_flops_of_the_mars_model():
    # the linearisation dominates (four RK4 stages of a 7 x 10 tangent product), and the
    # total stays within the scope table's ~8 kflop per node and SCP iteration
    f = bench.flops_per_node_scp(7, 3, bench.MARS7_F_FLOPS)
    assert f == 7249
    assert 6000 <= f <= 9000
    assert bench.flops_per_node_scp(7, 3, 0) < f   # the model evaluations are counted
    assert bench.flops_per_node_iter(7, 3, bench.mars_mirror_flops()) == 1206
