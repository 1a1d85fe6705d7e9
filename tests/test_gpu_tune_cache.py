"""Persistent tuner cache (DSRG_TUNE_CACHE): the first process times tile
and route candidates and appends its decisions to the file; a second
process reads them, times nothing new (the file is unchanged) and, using the
same choices, returns bit-identical energies."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHILD = r"""
import json, sys
sys.path.insert(0, %r)
import synth, paper_1701_02011_gb300 as g
inst = synth.make_instance(2, 4, 4, 30, 120, 0.5, seed=5)
h = g.Dsrg(inst, precision=g.DSRG_PREC_SPLIT, slices=6, tune=True)
print(json.dumps(h.pt3()))
h.close()
""" % ROOT


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_02011_gb300 import build
    build.build()


def _run(path):
    env = dict(os.environ, DSRG_TUNE_CACHE=path)
    out = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_decisions_persist_across_processes(lib, tmp_path):
    path = str(tmp_path / "tune.txt")
    e1 = _run(path)
    text1 = open(path).read()
    kinds = {line.split()[0] for line in text1.splitlines()}
    assert "tile" in kinds, text1
    e2 = _run(path)
    assert open(path).read() == text1   # nothing timed again
    assert e1 == e2
