"""Host-side parts of bench.py (no GPU): the ncu traffic record and the
reference arm's JSON line (the oracle timed on the host cores)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

CSV = '''==PROF== Connected to process 1
"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"
"0","1","python3","h","void mxp::k_persist2d_x2<float2, 6, 48, 8, 14, 2, 0>(PersistArgs)","1","7","(384, 1, 1)","(143, 1, 1)","0","10.3","m","dram__bytes_read.sum","byte","18000000"
"0","1","python3","h","void mxp::k_persist2d_x2<float2, 6, 48, 8, 14, 2, 0>(PersistArgs)","1","7","(384, 1, 1)","(143, 1, 1)","0","10.3","m","dram__bytes_write.sum","byte","900000"
"0","1","python3","h","void mxp::k_persist2d_x2<float2, 6, 48, 8, 14, 2, 0>(PersistArgs)","1","7","(384, 1, 1)","(143, 1, 1)","0","10.3","m","gpu__time_duration.sum","ns","4100000"
"1","1","python3","h","void mxp::k_step<float2, 2, 1, 0>(Geom)","1","7","(128, 1, 1)","(9, 1088, 1)","0","10.3","m","dram__bytes_read.sum","byte","5"
'''


def test_record_traffic_sums_read_and_write_of_the_named_kernel(tmp_path):
    csv_path = tmp_path / "t.csv"
    csv_path.write_text(CSV)
    out = tmp_path / "traffic.json"
    bench.record_traffic("persist2d", "c64", str(csv_path), str(out))
    rec = json.loads(out.read_text())["persist2d:c64"]
    assert rec["dram_bytes_per_launch"] == 18900000.0 and rec["launches"] == 1
    assert rec["kernel_sha"] == bench.kernel_hash("persist2d")


def test_record_traffic_rejects_scaled_units(tmp_path):
    csv_path = tmp_path / "t.csv"
    csv_path.write_text(CSV.replace('"byte","18000000"', '"Mbyte","18.0"'))
    with pytest.raises(SystemExit):
        bench.record_traffic("persist2d", "c64", str(csv_path), str(tmp_path / "x.json"))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
