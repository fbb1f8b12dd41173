"""CPU-side checks of the C-ABI library: it builds, loads, exports every entry point
declared in include/fmdp.h, its ctypes structures match the C layout, and it refuses
to run without a GPU (no CPU fallback). No compute call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2008_03518_gb300 import build, fmdp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fmdp.h")


def header_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fmdp_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return fmdp.load()


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert len(names) >= 20
    assert sorted(fmdp.EXPORTS) == names
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (fmdp_\w+)", out))
    for n in names:
        assert n in exported, n
        assert getattr(lib, n) is not None


def test_struct_layouts_match_header_sizes():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "fmdp.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(fmdp_airspace), sizeof(fmdp_action),
         sizeof(fmdp_sep), sizeof(fmdp_well), sizeof(fmdp_options), sizeof(fmdp_request), sizeof(fmdp_result),
         sizeof(fmdp_sep_report), sizeof(fmdp_stats), sizeof(fmdp_serve_options), sizeof(fmdp_serve_report),
         sizeof(fmdp_learned_report), sizeof(fmdp_tune_entry), sizeof(fmdp_tune_report));
  printf("%zu %zu %zu\n", offsetof(fmdp_result, xyz), offsetof(fmdp_request, depart_step), offsetof(fmdp_airspace, static_wells));
  return 0;
}'''
    import tempfile
    d = tempfile.mkdtemp()
    c = os.path.join(d, "sz.c")
    open(c, "w").write(src)
    exe = os.path.join(d, "sz")
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
    sizes, offs = [list(map(int, line.split())) for line in subprocess.run([exe], capture_output=True, text=True).stdout.splitlines()]
    py = [ctypes.sizeof(t) for t in (fmdp.Airspace, fmdp.Action, fmdp.Sep, fmdp.Well, fmdp.Options, fmdp.Request,
                                     fmdp.Result, fmdp.SepReport, fmdp.Stats, fmdp.ServeOptions,
                                     fmdp.ServeReport, fmdp.LearnedReport, fmdp.TuneEntry, fmdp.TuneReport)]
    assert py == sizes
    assert offs == [fmdp.Result.xyz.offset, fmdp.Request.depart_step.offset, fmdp.Airspace.static_wells.offset]


def test_options_default_is_the_paper_setting(lib):
    o = fmdp.Options()
    lib.fmdp_options_default(ctypes.byref(o))
    assert o.combine == 0 and o.n_wells == 0 and o.goal_reward == 200.0 and o.lookahead_W == 1


def test_null_arguments_are_rejected_without_a_device(lib):
    assert lib.fmdp_create(None, 0.99, None, 0, None, None, None) == -1
    h = ctypes.c_void_p()
    assert lib.fmdp_create(None, 0.99, None, 0, None, None, ctypes.byref(h)) == -1
    assert h.value is None
    assert lib.fmdp_schedule(None, None, None) == -1
    assert lib.fmdp_add_plan(None, 0, None, 0, None) == -1
    assert lib.fmdp_save_plans(None, b"x", None) == -1
    assert lib.fmdp_load_plans(None, b"x", None, 0, None) == -1


def test_metrics_lines_are_plain_json(tmp_path):
    """append_jsonl writes one JSON line per record, numpy values as plain numbers."""
    import json

    import numpy as np

    p = tmp_path / "m.jsonl"
    fmdp.append_jsonl(str(p), {"a": np.int64(3), "b": np.arange(3, dtype=np.float32), "c": {"d": np.float64(0.5)}})
    fmdp.append_jsonl(str(p), {"a": 4})
    lines = p.read_text().splitlines()
    assert [json.loads(x) for x in lines] == [{"a": 3, "b": [0.0, 1.0, 2.0], "c": {"d": 0.5}}, {"a": 4}]


def test_no_cpu_fallback_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2008_03518_gb300 import scenarios as S
    sc = S.c1_plain_small()
    with pytest.raises(fmdp.FmdpError) as e:
        fmdp.Scheduler.from_scenario(sc)
    assert e.value.status == -3  # FMDP_ERR_CUDA: no device, and nothing runs on the CPU


def test_vectorised_request_and_result_marshalling():
    """Requests converted column by column equal the record-by-record conversion byte for
    byte; result buffers are named per request and read back as views."""
    import numpy as np
    from paper_2008_03518_gb300 import scenarios as S

    reqs = S.c1_plain_small().requests
    n = len(reqs)
    fast = fmdp._requests(reqs)
    slow = (fmdp.Request * n)(*[fmdp.make_request(r) for r in reqs])
    assert bytes(fast) == bytes(slow)
    as_dicts = [{k: reqs[k][i] for k in reqs.dtype.names} for i in range(3)]
    assert bytes(fmdp._requests(as_dicts)) == bytes(slow)[: 3 * ctypes.sizeof(fmdp.Request)]

    res = (fmdp.Result * 4)()
    xyz, acts = fmdp._point_buffers(res, 4, 7)
    for i in range(4):
        assert ctypes.cast(res[i].xyz, ctypes.c_void_p).value == xyz[i].ctypes.data
        assert ctypes.cast(res[i].actions, ctypes.c_void_p).value == acts[i].ctypes.data
        res[i].verdict, res[i].n_points, res[i].plan_id = i - 1, i + 1, (1 << 63) + i
        res[i].min_sep_h = 0.5 * i
    xyz[2, :3] = 7.0
    out = fmdp._results(res, 4, xyz, acts)
    assert [d["verdict"] for d in out] == [-1, 0, 1, 2]
    assert [d["plan_id"] for d in out] == [(1 << 63) + i for i in range(4)]
    assert out[3]["min_sep_h"] == 1.5 and out[2]["xyz"].shape == (3, 3) and (out[2]["xyz"] == 7.0).all()
    assert out[0]["actions"].shape == (0,) and out[3]["actions"].shape == (3,)
    assert set(out[0]) == {f for f, _ in fmdp.Result._fields_}


def test_packed_plans_reject_mismatched_arrays_before_any_call():
    """add_plans_packed checks its arrays on the host (one t0 and one count per plan, three
    values per sample) before it reaches the library."""
    import numpy as np

    s = object.__new__(fmdp.Scheduler)  # no device context: the checks come first
    s._L, s._h = None, None
    with pytest.raises(ValueError):
        fmdp.Scheduler.add_plans_packed(s, [0, 5], [3], np.zeros((3, 3), np.float32))
    with pytest.raises(ValueError):
        fmdp.Scheduler.add_plans_packed(s, [0], [3], np.zeros((2, 3), np.float32))
    with pytest.raises(ValueError):
        fmdp.Scheduler.add_plans_packed(s, [[0]], [[3]], np.zeros((3, 3), np.float32))
    assert fmdp.Scheduler.add_plans_packed(s, [], [], np.zeros((0, 3), np.float32)).size == 0


def test_q_eval_figure_of_the_bench():
    """The bench's q_eval figure: the well scan's operations as the kernel performs them
    (20 FP32 + 1 MUFU per sample culled, 7 FP32 per well of a sample inside the cull radius,
    10 FP32 + 1 MUFU per (sample, reachable well) pair and action) over the rollout kernel's
    time, against the rates the device probe measured."""
    import sys as _sys

    _sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    kt = dict(rollout_steps=1000, qe_items=40_000, qe_near=3_000, qe_wells=1_000)
    peaks = dict(fp32_tflops=80.0, mufu_rsqrt_tops=5.0, sm_mhz=2000.0)
    q = bench.q_eval_counted(kt, 25, 5, peaks, 1900.0, 2.0)
    assert q["bound"] == "alu"
    fp32 = 20 * 40_000 + 7 * 5 * 3_000 + 10 * 25 * 1_000
    mufu = 40_000 + 25 * 1_000
    assert q["counted"]["fp32_ops"] == fp32 and q["counted"]["mufu_ops"] == mufu
    assert q["fp32"]["achieved"] == pytest.approx(fp32 / 2e-3 / 1e12)
    assert q["fp32"]["frac"] == pytest.approx(q["fp32"]["achieved"] / 80.0)
    assert q["mufu"]["frac"] == pytest.approx(mufu / 2e-3 / 1e12 / 5.0)
    assert bench.q_eval_counted(dict(kt, qe_items=0), 25, 5, peaks, None, 2.0) is None
    assert bench.q_eval_counted(kt, 25, 5, None, None, 2.0) is None
