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


def test_traffic_entries_are_per_launch_byte_counts():
    """The roofline block's `traffic` entries are DRAM bytes of one kernel on one workload:
    positive numbers, keyed by (workload, kernel), nothing else."""
    sys.path.insert(0, ROOT)
    import bench
    for key, v in bench.TRAFFIC.items():
        assert isinstance(key, tuple) and len(key) == 2, key
        assert key[0] in bench.SMAX, key
        assert key[1].startswith("k_"), key
        assert v is None or (isinstance(v, float) and v > 0), (key, v)


def test_error_vs_oracle_fields():
    """The per-result error entry on a tiny case where the GPU side is replaced by the
    oracle's own answer (zero error) and by a perturbed copy (outside the tolerances)."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    import oracle
    from paper_1302_5010_gb300 import synth
    P = synth.small_problem(64, 128, 3, 3, 6, rho=2, seed=5, lam_frac=0.05)
    Xo, _ = oracle.bmpl(P.At, P.B, P.lam, P.rho)
    e = bench.error_vs_oracle(P, Xo.copy(), Xo)
    assert e["signals"] == 3 and e["within"] and e["rel_objective_max"] == 0.0 and e["x_rel_fro"] == 0.0
    bad = Xo.copy()
    j = int(np.argmax(np.abs(bad[0])))
    bad[0, j] *= 1.5
    bad[1, (j + 1) % P.m] += 0.5 * np.abs(Xo[1]).max()
    e = bench.error_vs_oracle(P, bad, Xo)
    assert not e["within"] and e["support_mismatch_signals"] >= 1 and e["x_rel_fro"] > 1e-4
