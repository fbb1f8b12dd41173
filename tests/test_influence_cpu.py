"""The pipelined engine's influence test (csrc/pipe_influence.cuh: first_influenced, which
skips steps by chunk and group bounding boxes and by the table-operation counts each chunk
read) against the same rule taken step by step, over random flights with and without
encounters (tests/influence_check.cpp). A step the boxes skipped wrongly would let a plan
that an earlier admission changed stand. Runs on the host: g++ only, no GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2008_03518_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path_factory.mktemp("influence") / "influence_check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-Wall", "-Werror", "-I", CSRC,
                    os.path.join(HERE, "influence_check.cpp"), "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_box_skipping_never_misses_an_influenced_step(checker, seed):
    r = subprocess.run([checker, str(seed), "40000"], capture_output=True, text=True)
    out = r.stdout.split()
    assert r.returncode == 0 and out[0] == "ok", r.stdout + r.stderr
    hits, seps, clear = map(int, out[1:])
    # the cases cover every outcome: influenced steps, verdict flags and no influence
    assert hits > 1000 and seps > 500 and clear > 1000
