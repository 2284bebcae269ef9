"""Host-side accounting of bench.py (no GPU): the algorithmic bytes of the
roofline under both pass schedules, and the keying of profiled DRAM traffic
to the kernel sources."""
import json
import os

import bench


def test_pass_units_match_the_pass_flags():
    """Q-vectors per pixel of each pass (one iteration, and the first and
    last of two): C, the old messages once written, the new ones when read."""
    assert [bench.pass_units(p, 0, 1) for p in range(4)] == [(2, False), (4, False), (4, False), (3, True)]
    assert [bench.pass_units(p, 0, 2)[0] for p in range(4)] == [2, 4, 4, 5]
    assert [bench.pass_units(p, 1, 2)[0] for p in range(4)] == [4, 5, 4, 3]


def test_paired_launch_bytes_are_the_sum_of_their_passes():
    W, H, Q = 45, 37, 64
    for iters in (1, 2, 3):
        single = bench.launch_bytes(4 * iters, W, H, Q, iters)
        paired = bench.launch_bytes(2 * iters, W, H, Q, iters)
        assert len(single) == 4 * iters and len(paired) == 2 * iters
        assert sum(single) == sum(paired)
        for i in range(2 * iters):
            assert paired[i] == single[2 * i] + single[2 * i + 1]
    # one iteration: 13 Q-vectors per pixel plus the labels
    assert sum(bench.launch_bytes(2, W, H, Q, 1)) == 13 * W * H * Q * 4 + W * H * 4


def test_kernel_hash_ignores_comments_only():
    code = "int f(int a) {\n    return a + 1;  // add one\n}\n/* note */\n"
    same = "// header\nint f(int a) {\n\n    return a + 1;\n}\n"
    other = "int f(int a) {\n    return a + 2;\n}\n"
    assert bench._code_only(code) == bench._code_only(same)
    assert bench._code_only(code) != bench._code_only(other)


def test_profiled_traffic_is_keyed_to_the_current_sources():
    """Every committed traffic entry names its kernel and matches the hash of
    the sources in the tree (or the bench line reports traffic as null)."""
    path = os.path.join(bench.ROOT, "profiles", "edp_pass_traffic.json")
    entries = json.load(open(path))
    assert entries
    for workload, e in entries.items():
        assert workload in bench.WORKLOADS
        assert e["kernel"] in bench.KERNEL_SOURCES
        got = bench.profiled_traffic(workload, e["kernel"])
        if e["source_hash"] == bench.kernel_source_hash(e["kernel"]):
            assert got == float(e["dram_bytes_per_launch"])
        else:
            assert got is None
        assert bench.profiled_traffic(workload, "no_such_kernel") is None
