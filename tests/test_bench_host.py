"""Host-side helpers of bench.py (no GPU): the kernel-source hash that keys the ncu traffic
counters ignores comments and layout but not code, and the committed profile lines parse."""
import bench


def test_code_only_strips_comments_keeps_literals():
    src = 'int a = 1; // note\n/* block\n comment */ asm volatile("// kept" ::: "memory"); char c = \'/\';'
    assert bench.code_only(src) == 'int a = 1; asm volatile("// kept" ::: "memory"); char c = \'/\';'
    assert bench.code_only("a  =\n\t b;") == bench.code_only("a = b;")
    assert bench.code_only("a = b;") != bench.code_only("a = c;")


def test_profiled_traffic_matches_current_sources():
    # the committed counters were taken on the current kernel code
    t = bench.profiled_traffic("k_stream_collide<D2Q37,fp32,periodic>")
    assert t is not None and 9.0e9 < t < 1.1e10      # ~592 B x 4096^2 cells
