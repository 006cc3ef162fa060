"""Host-side pieces of bench.py that the reported numbers rest on: the
algorithmic bytes of the roofline (the per-unit figures the design states,
times the units of the 24 h workload) and the rule that a measured DRAM
traffic is reported only while the screen's sources hash to the ones it was
captured on."""
import hashlib
import os

import bench


def test_traversal_algorithmic_bytes_of_the_24h_screen():
    # units of the 24 h, n = 16848 screen: boxes, merged pairs (run starts)
    # and runs of more than one cell (one end record each)
    m = {"boxes": 17392488, "records": 163639734, "open_runs": 28002408, "morton_bits": 10,
         "T": 86400}
    b = bench.algorithmic_bytes(m, 16848)
    N = m["boxes"]
    # per sorted box 32 (box) + 8 (object id, neighbour positions), per node
    # 40, per record 8
    assert b["traverse"] == N * 40 + (N - 1) * 40 + (m["records"] + m["open_runs"]) * 8
    assert b["traverse"] == 2924536136
    # boxes: elements in, box (32 B), object id, box id and the 40-bit key out
    assert b["boxes"] == 56 * 16848 + N * (32 + 4 + 4 + 8)


def test_measured_traffic_follows_the_screen_sources():
    path = os.path.join(bench.ROOT, "profiles", "k_traverse2_catalog16848_24h.md")
    fields = dict(line.split(":", 1) for line in open(path)
                  if line.split(":", 1)[0] in ("traffic_bytes_per_launch", "source_sha256"))
    h = hashlib.sha256()
    for f in bench.library_sources():
        h.update(open(f, "rb").read())
    t = bench.measured_traffic("catalog24h")
    if fields["source_sha256"].strip() == h.hexdigest()[:16]:
        assert t == float(fields["traffic_bytes_per_launch"])
    else:
        assert t is None
    # only the default workloads' traversal was captured
    assert bench.measured_traffic("band_slab") is None
    # the narrow phase and the refinement are not screen sources
    names = [os.path.basename(f) for f in bench.library_sources()]
    assert "narrow.cu" not in names and "refine.cu" not in names and "traverse.cu" in names
