"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps
the one-JSON-line contract, on the CPU: the keys, their types, the metric
and config of the device arm, and only rank 0 printing under several ranks.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2",
                          "--warmup", "0", "--cpu-sample", "64"], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return [ln for ln in out.stdout.splitlines() if ln.strip()]


def test_reference_arm_prints_one_contract_line():
    lines = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "converged POI/s" and d["unit"] == "POI/s"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 0
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["vs_baseline"] is None and d["dtype"] == "f64"
    assert d["config"]["workload"] == "affine1024" and d["config"]["pois_per_pair"] == 36100
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["sample"].startswith("64 evenly spaced POIs")
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_traffic_record_from_ncu_csv(tmp_path):
    """bench.py --traffic-record sums dram read + write per captured launch of
    the matching kernel and stores the sources' hashes as they are when it
    runs (in the capture's own command)."""
    import hashlib
    import json
    import subprocess
    import sys
    csv = tmp_path / "t.csv"
    hdr = '"ID","Process ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n'
    rows = [
        '"0","1","subpixel_kernel<false>(dic::SubpixelParams)","dram__bytes_read.sum","Mbyte","20.50"\n',
        '"0","1","subpixel_kernel<false>(dic::SubpixelParams)","dram__bytes_write.sum","byte","1,000"\n',
        '"1","1","tile_kernel(dic::SearchTcParams)","dram__bytes_read.sum","Mbyte","99.00"\n',
        '"2","1","subpixel_kernel<false>(dic::SubpixelParams)","dram__bytes_read.sum","Mbyte","20.70"\n',
        '"2","1","subpixel_kernel<false>(dic::SubpixelParams)","dram__bytes_write.sum","byte","3,000"\n',
    ]
    csv.write_text("==PROF== noise line\n" + hdr + "".join(rows))
    out = tmp_path / "rec.json"
    src = "paper_1905_06228_gb300/csrc/k_subpixel.cu"
    subprocess.check_call([sys.executable, os.path.join(ROOT, "bench.py"), "--traffic-record",
                           str(csv), "--kernel", "subpixel_kernel", "--sources", src,
                           "--out", str(out), "--command", "ncu ..."], cwd=ROOT,
                          stdout=subprocess.DEVNULL)
    rec = json.loads(out.read_text())
    assert rec["launches"] == 2
    assert rec["bytes_per_launch"] == int(round((20.5e6 + 1000 + 20.7e6 + 3000) / 2))
    want = hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest()
    assert rec["sources"][src] == want
