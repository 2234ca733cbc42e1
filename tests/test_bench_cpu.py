"""bench.py's CPU-side legs (no GPU): the reference arm's JSON line and the oracle's full-size
step-time model."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_full_size_model_reduces_to_the_sample():
    import bench
    sample = {"nodes": 1000, "cells": [10, 10, 10], "s_per_step": 2.0,
              "it_per_step": {"ms": 10.0, "mech": 20.0, "gs": 30.0},
              "s_per_iteration": {"ms": 0.01, "mech": 0.02, "gs": 0.005}}
    # same size, measured counts = the sample's: the sample's own step time
    t, its, _ = bench.oracle_full_size_model(sample, 1000, (10, 10, 10), sample["it_per_step"])
    assert t == pytest.approx(2.0, rel=1e-12)
    # twice the nodes and twice the linear size: non-CG time and iteration cost scale with the
    # nodes, K^ms / K^mech iterations with the linear size, GSPM iterations stay
    t2, its2, _ = bench.oracle_full_size_model(sample, 2000, (20, 10, 10))
    cg = 10 * 0.01 + 20 * 0.02 + 30 * 0.005
    expect = (2.0 - cg) * 2 + (20 * 0.01 + 40 * 0.02 + 30 * 0.005) * 2
    assert t2 == pytest.approx(expect, rel=1e-12)
    assert its2 == {"ms": 20.0, "mech": 40.0, "gs": 30.0}


@pytest.mark.slow
def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600, env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "steps/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
