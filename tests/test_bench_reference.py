"""bench.py's reference arm (the FP64 CPU oracle timed on the host cores, each
step a sample of the workload's elements taken as a mesh of its own) runs
without a GPU and prints one JSON line of the benchmark's contract."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_its_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "beam16", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, cwd=ROOT,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["unit"] == "pairs/s" and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_work_shape_option_is_parsed_and_checked():
    """--work-shape takes four integers (clip block, PCG rows per block, PCG
    cluster, rows per block of the captured step's solve); anything else is a
    usage error before any work starts."""
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path.pop(0)
    argv = sys.argv
    try:
        sys.argv = ["bench.py", "--work-shape", "64,64,0,128"]
        assert bench.parse().work_shape == (64, 64, 0, 128)
        sys.argv = ["bench.py"]
        assert bench.parse().work_shape is None
    finally:
        sys.argv = argv
    for bad in ("64,64,0", "64,x,0,64", "64,64,0,64,4,1"):
        out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--work-shape", bad],
                             capture_output=True, text=True, cwd=ROOT, timeout=120)
        assert out.returncode == 2, (bad, out.stderr[-500:])
