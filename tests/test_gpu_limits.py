"""Parity at the limits of the boundary: 32 actions (every lane of a warp is an action),
8 wells per plan (the largest well table), the largest lookahead window (16 sub-steps with
32 actions: 512 (action, sub-step) pairs per step), 64 static wells, and a plan table whose
slot count is not a multiple of the tile sizes. Each case runs the GPU against the FP64
oracle: action values within 1e-5 of the term scale, trajectories bit for bit (the oracle
follows the GPU at near-ties), identical verdicts.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import ADMITTED, Oracle  # noqa: E402
from paper_2008_03518_gb300 import scenarios as S  # noqa: E402
from paper_2008_03518_gb300.fmdp import Scheduler  # noqa: E402
from tests.parity_util import fcfs_parity  # noqa: E402

BOX = (0.0, 0.0, 0.0, 10000.0, 10000.0, 500.0)
# 8 headings (multiples of 15 degrees) x 4 climb rates = 32 actions
ACT32 = [(float(h), float(c)) for h in (-60, -45, -30, -15, 0, 15, 30, 45) for c in (-3.0, -1.0, 1.0, 3.0)]
# 8 wells: the paper's five (Table 3) and three more along the same rule
WELLS8 = tuple((float(t), 300.0 + 10.0 * t, 1000.0, 0.97) for t in (-10, -5, 0, 5, 10, 15, 20, 25))


def _traffic(seed, n_plans=150, n_req=6, max_slots=173):
    rng = np.random.default_rng(seed)
    plans = S.straight_plans(rng, BOX, n_plans, 50.0, 450.0, 20.0, 40.0, 0, 400, 1.0)
    reqs = S.make_requests(rng, BOX, n_req, zlo=60.0, zhi=440.0, tlo=0, thi=300, horizon=900)
    return plans, reqs, max_slots


def _pair(plans, max_slots, **kw):
    s = Scheduler(BOX, 1.0, 0.99, ACT32, (150.0, 30.0), n_slices_window=2048, max_slots=max_slots, **kw)
    o = Oracle(BOX, 1.0, 0.99, ACT32, (150.0, 30.0), **kw)
    for pl in plans:
        s.add_plan(pl.t0, pl.xyz)
        o.add_plan(pl.t0, pl.xyz)
    return s, o


@pytest.mark.parametrize("combine", [0, 1])
def test_32_actions_and_8_wells(combine):
    plans, reqs, max_slots = _traffic(201)
    s, o = _pair(plans, max_slots, wells=WELLS8, combine=combine)
    with s:
        verdicts, followed, steps = fcfs_parity(s, o, reqs, trace_q=True)
    assert steps > 500 and ADMITTED in verdicts


def test_largest_window_with_32_actions():
    plans, reqs, max_slots = _traffic(202, n_req=3)
    s, o = _pair(plans, max_slots, lookahead_W=16)
    with s:
        verdicts, followed, steps = fcfs_parity(s, o, reqs, trace_q=True)
    assert steps > 200


def test_64_static_wells():
    plans, reqs, max_slots = _traffic(203, n_plans=60, n_req=4)
    rng = np.random.default_rng(7)
    sw = np.stack([rng.uniform(500, 9500, 64), rng.uniform(500, 9500, 64), rng.uniform(50, 450, 64),
                   rng.uniform(100, 400, 64), np.full(64, 1000.0), np.full(64, 0.99)], axis=1)
    s, o = _pair(plans, max_slots, static_wells=sw)
    with s:
        verdicts, followed, steps = fcfs_parity(s, o, reqs, trace_q=True)
    assert steps > 200
