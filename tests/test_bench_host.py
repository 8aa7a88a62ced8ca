"""Host-side parts of bench.py that need no GPU: the algorithmic-bytes model
(the roofline numerator), the ncu capture digest and the DRAM traffic table
the roofline line reads."""
import json

import bench


def test_algorithmic_bytes_follow_the_per_source_model():
    # per source: 2m level probes + 8 B sigma per DAG arc + 9 B per vertex
    # (forward); 2m + 4 B c per arc + 13 B per vertex (backward); plus the
    # per-batch CSR and BC terms
    n, m, a, nsrc, B = 1000, 5000, 30000, 256, 256
    fwd, bwd = bench.algorithmic_bytes(n, m, a, nsrc, B)
    assert fwd == nsrc * (2 * m + 9 * n) + 8 * a + 1 * (8 * m + 4 * n)
    assert bwd == nsrc * (2 * m + 13 * n) + 4 * a + 1 * (8 * m + 4 * n + 16 * n)
    fwd2, bwd2 = bench.algorithmic_bytes(n, m, a, 2 * nsrc, B)
    assert fwd2 > fwd and bwd2 > bwd  # more sources, more bytes; two batches pay the CSR twice


def test_code_text_ignores_comments_and_space():
    a = "int x = 1; // one\n/* block\n comment */ float  y;\n"
    b = "int x=1;\nfloat y;   // other words\n"
    assert bench.code_text(a) == bench.code_text(b)
    assert bench.code_text(a) != bench.code_text("int x = 2; float y;")


def test_traffic_table_from_an_ncu_csv(tmp_path):
    hdr = '"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n'
    rows = [
        ('0', 'void unnamed>::k_forward<1, false>(MsParams, int)', 'dram__bytes_read.sum', 'byte', '5000'),
        ('1', 'void unnamed>::k_forward<8, false>(MsParams, int)', 'dram__bytes_read.sum', 'byte', '1000'),
        ('1', 'void unnamed>::k_forward<8, false>(MsParams, int)', 'dram__bytes_write.sum', 'byte', '200'),
        ('1', 'void unnamed>::k_forward<8, false>(MsParams, int)', 'gpu__time_duration.sum', 'ns', '5000'),
        ('2', 'void unnamed>::k_first<8>(MsParams)', 'dram__bytes_read.sum', 'byte', '30'),
        ('2', 'void unnamed>::k_first<8>(MsParams)', 'dram__bytes_write.sum', 'byte', '10'),
        ('3', 'void unnamed>::k_backward<8, false>(MsParams, int)', 'dram__bytes_read.sum', 'byte', '700'),
        ('3', 'void unnamed>::k_backward<8, false>(MsParams, int)', 'dram__bytes_write.sum', 'byte', '100'),
        ('4', 'void unnamed>::k_backward<8, false>(MsParams, int)', 'dram__bytes_read.sum', 'byte', '1,300'),
    ]
    csv_path = tmp_path / "t.csv"
    csv_path.write_text("==PROF== noise\n" + hdr + "".join(",".join(f'"{x}"' for x in r) + "\n" for r in rows))
    out_path = tmp_path / "traffic.json"
    out = bench.write_traffic(str(csv_path), "cmd", out_path=str(out_path), echo=False)
    # the 32-wide landmark pass is left out; per launch of each kind
    assert out["kinds"]["forward"]["launches"] == 2
    assert out["kinds"]["forward"]["dram_bytes_per_launch"] == 620.0
    assert out["kinds"]["backward"]["dram_bytes_per_launch"] == 1050.0
    assert abs(out["kinds"]["forward"]["ncu_time_ms"] - 0.005) < 1e-12
    assert bench.measured_traffic("backward", path=str(out_path)) == 1050.0
    doc = json.loads(out_path.read_text())
    doc["csrc_sha256"] = "0" * 64
    out_path.write_text(json.dumps(doc))
    assert bench.measured_traffic("backward", path=str(out_path)) is None


def test_committed_traffic_table_is_well_formed():
    # the table names the kernel sources it was taken on; when they have
    # changed since, the bench reports traffic as null rather than stale bytes
    with open(bench.TRAFFIC_JSON) as f:
        doc = json.load(f)
    assert len(doc["csrc_sha256"]) == 64 and doc["command"]
    assert set(doc["kinds"]) >= {"forward", "backward", "hash"}
    got = bench.measured_traffic("forward")
    assert (got is None) == (doc["csrc_sha256"] != bench.csrc_digest())


def test_grid_traffic_table_from_an_ncu_csv(tmp_path):
    hdr = '"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n'
    rows = [
        ('0', 'void unnamed>::k_map_ids(const int *, const int *, int *, int)', 'dram__bytes_read.sum', 'byte', '99'),
        ('1', 'void unnamed>::k_wsssp_packed<512>(WParams)', 'dram__bytes_read.sum', 'byte', '3,000'),
        ('1', 'void unnamed>::k_wsssp_packed<512>(WParams)', 'dram__bytes_write.sum', 'byte', '1000'),
        ('1', 'void unnamed>::k_wsssp_packed<512>(WParams)', 'gpu__time_duration.sum', 'ns', '2000000'),
    ]
    csv_path = tmp_path / "g.csv"
    csv_path.write_text(hdr + "".join(",".join(f'"{x}"' for x in r) + "\n" for r in rows))
    out_path = tmp_path / "grid.json"
    out = bench.write_traffic_grid(str(csv_path), 8, "cmd", out_path=str(out_path))
    assert out["launches"] == 1 and out["dram_bytes_per_source"] == 500.0
    assert abs(out["ncu_time_ms"] - 2.0) < 1e-12
    assert bench.measured_traffic_grid(path=str(out_path)) == 500.0
    doc = json.loads(out_path.read_text())
    doc["csrc_sha256"] = "0" * 64
    out_path.write_text(json.dumps(doc))
    assert bench.measured_traffic_grid(path=str(out_path)) is None


def test_committed_grid_traffic_is_well_formed():
    with open(bench.TRAFFIC_GRID_JSON) as f:
        doc = json.load(f)
    assert len(doc["csrc_sha256"]) == 64 and doc["command"] and doc["sources"] > 0
    assert doc["dram_bytes_per_source"] == (doc["dram_read_bytes"] + doc["dram_write_bytes"]) / doc["sources"]
    got = bench.measured_traffic_grid()
    assert (got is None) == (doc["csrc_sha256"] != bench.csrc_digest(bench.GRID_SOURCES))
