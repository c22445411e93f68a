"""The bench's reference arm (the oracle on the host cores) on a small case:
one JSON line with the GPU arm's metric, unit and config keys, its value in
the metric's own definition (the step's bytes times the fraction of the
circuit's gates applied per second)."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line(svlib):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "14",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GB/s" and line["higher_is_better"] is True
    cfg = line["config"]
    for k in ("workload", "n_qubits", "layers", "gates", "fuse_max_k", "block_mode", "fused_blocks",
              "passes_per_step", "l2", "parallelism"):
        assert k in cfg, k
    n, npasses, ng = cfg["n_qubits"], cfg["passes_per_step"], cfg["gates"]
    step_bytes = (2 * npasses + 2) * 2 ** n * 8
    assert abs(line["value"] - line["gates_per_s"] * step_bytes / ng / 1e9) <= 1e-9 * max(1.0, line["value"])
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
