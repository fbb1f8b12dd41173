"""The plan table's host bookkeeping (csrc/plan_book.h: free slots in a two-level bitmap,
plans by slot with an ascending id list, expiry by last-step buckets of the window) against
ordered containers with the same meaning, over random admissions, roll-backs and expiries
(tests/plan_book_check.cpp). Runs on the host: g++ only, no GPU."""
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
    exe = str(tmp_path_factory.mktemp("plan_book") / "plan_book_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC,
                    os.path.join(HERE, "plan_book_check.cpp"), "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("seed,slots,window,rounds", [
    (1, 64, 32, 3000),        # a small table that fills up and empties often
    (2, 1000, 4096, 2000),    # slots that are not a multiple of 64, a wide window
    (3, 4160, 97, 3000),      # more than 64 words (two summary words), an odd window
    (4, 1, 8, 500),           # one slot
])
def test_plan_book_agrees_with_ordered_containers(checker, seed, slots, window, rounds):
    r = subprocess.run([checker, str(seed), str(slots), str(window), str(rounds)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
