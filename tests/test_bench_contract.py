"""The benchmark's reference arm (the FP64 oracle on the host cores) and its
JSON line, on CPU: the keys the line must carry and the single-rank behaviour."""
import contextlib
import io
import json
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    sys.path.insert(0, ROOT)
    import bench
    args = types.SimpleNamespace(config="c1", ref_signals=1, steps=2, warmup=1)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args, 0, 1)
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_metric_matches_baseline_file():
    sys.path.insert(0, ROOT)
    import bench
    with open(os.path.join(ROOT, "BASELINE.json")) as f:
        base = json.load(f)
    assert bench.METRIC == base["metric"]


def test_traffic_entries_name_committed_captures():
    """The roofline block's `traffic` comes from an ncu capture summarised under
    profiles/; each entry must name a summary that exists and quotes its command."""
    sys.path.insert(0, ROOT)
    import bench
    for kernel, entry in bench.TRAFFIC.items():
        if entry is None:
            continue
        assert entry["bytes_per_launch"] > 0, kernel
        path = entry["capture"].split()[0]
        assert path.startswith("profiles/"), kernel
        full = os.path.join(ROOT, path)
        assert os.path.isfile(full), path
        with open(full) as f:
            text = f.read()
        assert "ncu" in text and "--clock-control none" in text, path
