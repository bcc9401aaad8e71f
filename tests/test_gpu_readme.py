"""The Python example of README.md runs as written, through libnefty."""
import math
import pathlib
import re

import pytest

README = pathlib.Path(__file__).resolve().parents[1] / "README.md"


def _example() -> str:
    blocks = re.findall(r"```python\n(.*?)```", README.read_text(), re.S)
    assert len(blocks) == 1, "README.md holds one Python example"
    return blocks[0]


def test_readme_example_compiles():
    compile(_example(), str(README), "exec")


@pytest.mark.gpu
def test_readme_example_runs():
    ns = {}
    exec(compile(_example(), str(README), "exec"), ns)
    out, job = ns["out"], ns["job"]
    assert out["loss"] > 0 and math.isfinite(out["loss"])
    assert bool(out["grad_alpha"].isfinite().all())
    assert float(ns["field"].theta.grad.norm()) > 0
    assert ns["tv"] > 0
    assert job["state_name"] == "done" and job["status"] == 0 and job["iters_done"] == 3, job
    assert math.isfinite(job["loss"]) and job["loss"] > 0
