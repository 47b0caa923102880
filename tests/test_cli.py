"""The command line (python -m paper_2602_11734_gb300): argument handling on
the CPU; on the GPU, its files against the oracle-written 64^3 golden."""
import hashlib
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2602_11734_gb300 import __main__ as cli

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SMALL = ["--size", "64", "64", "64", "--solid-fraction", "0.7", "--cd", "0.002",
         "--g", "0.01", "0.0025", "0.000625", "--spacing", "0", "--seed", "1"]


def test_arguments_become_the_library_parameters():
    a = cli.parse(SMALL + ["--out", "x.raw", "--count", "1"])
    p = cli.params_of(a, 0)
    golden = json.loads(open(os.path.join(ROOT, "tests", "golden", "small_64.jsonl")).readline())
    for k, v in golden["params"].items():
        assert p[k] == v, k
    assert p["periodic"] == 0
    b = cli.parse(SMALL + ["--out", "r{i}.npy", "--count", "3", "--periodic", "--max-steps", "9"])
    assert [cli.params_of(b, k)["seed"] for k in range(3)] == [1, 2, 3]
    assert cli.params_of(b, 0)["periodic"] == 1 and cli.params_of(b, 0)["max_steps"] == 9


@pytest.mark.parametrize("bad", [
    ["--out", "x.raw"] + SMALL[:4] + SMALL[6:],                # no target
    SMALL + ["--target-count", "5", "--out", "x.raw"],         # two targets
    SMALL + ["--count", "2", "--out", "x.raw"],                # several files, one name
    SMALL + ["--count", "0", "--out", "x.raw"],
    SMALL + ["--packed", "--out", "x.npy"],
])
def test_invalid_arguments_are_rejected(bad):
    with pytest.raises(SystemExit):
        cli.parse(bad)


@pytest.mark.gpu
def test_cli_writes_the_oracle_realization(tmp_path):
    golden = json.loads(open(os.path.join(ROOT, "tests", "golden", "small_64.jsonl")).readline())
    out = tmp_path / "grain{i}.npy"
    r = subprocess.run([sys.executable, "-m", "paper_2602_11734_gb300", *SMALL, "--count", "2",
                        "--out", str(out)], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.strip().splitlines()]
    assert [x["seed"] for x in lines] == [1, 2]
    phase = np.load(tmp_path / "grain0.npy")
    assert phase.shape == (64, 64, 64) and phase.dtype == np.uint8
    assert hashlib.sha256(phase.tobytes()).hexdigest() == golden["sha256_u8"]
    assert lines[0]["solid_count"] == golden["solid_count"] == int(phase.sum())
    assert lines[0]["steps"] == golden["steps"]
    other = np.load(tmp_path / "grain1.npy")
    assert int(other.sum()) == lines[1]["solid_count"] == golden["target_count"]
    assert not np.array_equal(phase, other)
    # The packed grid of the same realization: bit x & 31 of word
    # (z * ny + y) * ceil(nx / 32) + x / 32.
    raw = tmp_path / "grain.raw"
    r = subprocess.run([sys.executable, "-m", "paper_2602_11734_gb300", *SMALL, "--packed",
                        "--out", str(raw)], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    words = np.fromfile(raw, dtype=np.uint32).reshape(64, 64, 2)
    bits = (words[..., :, None] >> np.arange(32, dtype=np.uint32)) & 1
    assert np.array_equal(bits.reshape(64, 64, 64).astype(np.uint8), phase)
