"""bench.py's command-line contract, on the host: the reference arm (the FP64
oracle on the host cores) prints one JSON line with the keys the contract
names, the other ranks of a multi-rank launch print nothing, and the native
arm fails loudly instead of falling back to the CPU when no GPU is present."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TINY = ["--nx", "24", "--ny", "20", "--nz", "6", "--nt", "8"]


def _run(args, env=None, timeout=300):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                          env=e, timeout=timeout, cwd=ROOT)


def test_reference_arm_line():
    res = _run(["--impl", "reference", "--steps", "2", "--warmup", "1", "--cpu-sample-steps", "2"] + TINY,
               env={"RANK": "0", "OMP_NUM_THREADS": "2"})
    assert res.returncode == 0, res.stderr
    lines = [ln for ln in res.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, res.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "fwd+adjoint Gcell-steps/s" and d["unit"] == "Gcell-steps/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["vs_baseline"] is None
    assert d["config"]["grid"] == [24, 20, 6] and d["config"]["nt"] == 8
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # value = cell-steps of the sampled steps / their time
    assert d["value"] == pytest.approx(24 * 20 * 6 * 2 / (d["ms_per_step"] / 1000.0) / 1e9, rel=1e-6)


def test_reference_arm_other_ranks_are_silent():
    res = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"] + TINY, env={"RANK": "1"})
    assert res.returncode == 0, res.stderr
    assert res.stdout.strip() == ""


def test_native_arm_fails_loudly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    res = _run(["--steps", "1", "--warmup", "3", "--no-cpu-baseline"] + TINY)
    assert res.returncode != 0
    assert '"value"' not in res.stdout
    assert "NEFTY_ECUDA" in res.stderr
