"""The autotuner's persistent table (no GPU needed): choices are kept under
keys of GPU name and shape in a flat JSON object at HIVC_TUNE_CACHE, read
once per process, merged and rewritten on every new choice."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SNIPPET = r"""
import ctypes, json, sys
sys.path.insert(0, {root!r})
from paper_2008_10273_gb300 import hivc
L = hivc.lib()
ops = json.loads(sys.argv[1])
out = []
for op in ops:
    if op[0] == "get":
        out.append(L.hivc_tune_lookup(op[1].encode()))
    else:
        out.append(L.hivc_tune_record(op[1].encode(), op[2]))
print(json.dumps(out))
"""


@pytest.fixture(scope="module")
def built():
    pytest.importorskip("torch")
    from paper_2008_10273_gb300 import build

    build.build()


def _run(path, ops):
    env = dict(os.environ, HIVC_TUNE_CACHE=str(path))
    r = subprocess.run([sys.executable, "-c", SNIPPET.format(root=ROOT), json.dumps(ops)], env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_choices_persist_across_processes(built, tmp_path):
    path = tmp_path / "sub" / "tune.json"  # the directory is created
    key = "NVIDIA GB300|coef|16384"
    assert _run(path, [["get", key], ["set", key, 2], ["get", key]]) == [-1, 0, 2]
    assert json.loads(path.read_text()) == {key: 2}
    # a new process starts with the file's choices and merges new ones
    assert _run(path, [["get", key], ["set", "g|sor|1920x1080", 0]]) == [2, 0]
    assert json.loads(path.read_text()) == {key: 2, "g|sor|1920x1080": 0}


def test_keys_with_quotes_and_a_malformed_file(built, tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{ not json")
    odd = 'gpu "x" \\ y|sor|3x3'
    assert _run(path, [["get", "a"], ["set", odd, 1], ["get", odd]]) == [-1, 0, 1]
    assert json.loads(path.read_text()) == {odd: 1}
    assert _run(path, [["get", odd], ["set", "", 1], ["set", "b", -1]]) == [1, -1, -1]
