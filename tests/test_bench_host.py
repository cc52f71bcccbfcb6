"""Host-side helpers of bench.py (no GPU): the kernel-source hash that keys the ncu traffic
counters ignores comments and layout but not code, and the committed profile lines parse."""
import bench


def test_code_only_strips_comments_keeps_literals():
    src = 'int a = 1; // note\n/* block\n comment */ asm volatile("// kept" ::: "memory"); char c = \'/\';'
    assert bench.code_only(src) == 'int a = 1; asm volatile("// kept" ::: "memory"); char c = \'/\';'
    assert bench.code_only("a  =\n\t b;") == bench.code_only("a = b;")
    assert bench.code_only("a = b;") != bench.code_only("a = c;")


def test_committed_traffic_line_parses():
    # a traffic line for the headline kernel is committed, in range (~592 B x 4096^2
    # cells); bench.py reports it only while its source hash matches the current code
    import glob
    import re
    pat = re.compile(r"traffic:\s*kernel=k_stream_collide<D2Q37,fp32,periodic>\s+src_sha=(\S+)\s+bytes_per_launch=(\d+)")
    hits = [m for f in glob.glob(bench.os.path.join(bench.ROOT, "profiles", "*.md")) for m in pat.finditer(open(f).read())]
    assert hits and all(9.0e9 < int(m.group(2)) < 1.1e10 for m in hits)
