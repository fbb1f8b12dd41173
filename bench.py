"""Benchmark: FCFS flight-plan scheduling throughput (scheduled plans/s) on GB300.

Workload (default): the 30 km x 30 km x 1 km airspace with a 512^2 fractal heightmap,
3000 seeded multi-leg known plans and 1000 FCFS requests with 25 actions and horizons up
to 1800 steps. One step = one whole FCFS pass: the plan table is restored to the 3000
known plans (device copy) and the 1000 requests are planned, checked and admitted in
arrival order on the GPU through pipelined speculative batches (one persistent rollout
launch fed by the host; results identical to planning them one after the other).
value = requests planned per second (admitted + rejected).

  value    : requests already resident in device memory, trajectories left on the device
  batch    : re-plans, resumed re-plans, rollout occupancy, per-request time to result
  roofline : the rollout kernel (dominant) against HBM; q_eval (its well scan) against the
             FP32 and MUFU rates measured on the device, its operations counted as performed
  modes    : sweep over 3k / 20k / 100k known plans (batched, waves, plain sequential and
             learned FCFS: plans/s and p50 / p99 time to result), the 20k separation check
             against HBM, serving at the 100k-plan table up to saturation, the MLP against
             bf16, departure candidates, the paper's lookahead window, co-simulation
  e2e      : through the C ABI with host buffers: known plans uploaded from host memory,
             requests uploaded, trajectories and verdicts copied back, every step
  cpu_baseline: the FP64 oracle on this host's cores (one thread and all of them), bounded

--impl reference runs the FP64 CPU oracle as the reference arm (rank 0 only).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "scheduled plans/s vs known-plan count (plain/batched/learned); p99 latency"
UNIT = "plans/s"


from paper_2008_03518_gb300.replicas import Replicas, dist_env  # noqa: E402


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.proc = None
        self.path = os.path.join(os.environ.get("FMDP_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"fmdp_clocks_{os.getpid()}.csv")
        self.index = index

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm), "reasons": sorted(reasons)}


def traffic_from_profile(kernel_src):
    """DRAM traffic per algorithmic byte recorded from an ncu capture, valid only while the
    kernel's source is unchanged (the profile records the source digest)."""
    digest = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", "rollout_kernel_c2.md")
    try:
        for line in open(path):
            if line.startswith("traffic_per_algorithmic_byte:"):
                parts = dict(kv.split("=") for kv in line.split(":", 1)[1].split())
                if parts.get("src") == digest:
                    return float(parts["value"])
    except OSError:
        pass
    return None


def q_eval_counted(kt, n_actions, n_wells, peaks_dev, sm_mhz_run, ms):
    """The well scan (q_eval) of the rollout kernel against the measured FP32 and MUFU
    rates, its operations counted as the kernel performs them: every plan sample a step
    reads is culled by one lane (offset, velocity, reach and distance: 20 FP32 operations and
    one MUFU reciprocal square root); a sample inside the cull radius gets its reachable-well
    mask (7 FP32 operations per well); each (sample, reachable well) pair is valued by every
    action's lane (centre offset and distance: 10 FP32 operations and one MUFU reciprocal
    square root). ms: the rollout kernel's summed duration over the counted steps."""
    items, near, wells = kt.get("qe_items", 0), kt.get("qe_near", 0), kt.get("qe_wells", 0)
    if items <= 0 or ms <= 0.0 or not peaks_dev:
        return None
    fp32 = 20.0 * items + 7.0 * n_wells * near + 10.0 * n_actions * wells
    mufu = 1.0 * items + 1.0 * n_actions * wells
    s = ms / 1e3
    f_ach, m_ach = fp32 / s / 1e12, mufu / s / 1e12
    f_peak, m_peak = peaks_dev["fp32_tflops"], peaks_dev["mufu_rsqrt_tops"]
    out = {"kernel": "rollout_kernel (q_eval: the well scan)", "bound": "alu",
           "fp32": {"achieved": f_ach, "peak": f_peak, "unit": "TFLOP/s", "frac": f_ach / f_peak},
           "mufu": {"achieved": m_ach, "peak": m_peak, "unit": "Top/s", "frac": m_ach / m_peak},
           "counted": {"items_culled": items, "items_inside_cull_radius": near, "sample_well_pairs": wells,
                       "fp32_ops": fp32, "mufu_ops": mufu, "rollout_steps": kt.get("rollout_steps", 0)},
           "peak_from": "fmdp_probe_peaks on this device: FFMA and MUFU rsqrt chains over all SMs "
                        f"(SM clock {peaks_dev['sm_mhz']:.0f} MHz during the probe)"}
    if sm_mhz_run:
        out["sm_mhz_run"] = sm_mhz_run
    return out


def cpu_baseline(sc, seconds=8.0):
    """The FP64 oracle, as it stands, on the first requests of the same workload: one thread,
    then every host core (a step's actions valued in parallel; same results)."""
    import oracle as O

    out = {}
    for label, threads in (("single", 1), ("multi", os.cpu_count() or 1)):
        used = O.set_threads(threads)
        o = O.Oracle.from_scenario(sc)
        n = 0
        t0 = time.perf_counter()
        while n < len(sc.requests) and (time.perf_counter() - t0) < seconds:
            o.schedule(sc.requests[n])
            n += 1
        dt = time.perf_counter() - t0
        out[label] = {"value": n / dt, "cores": used, "requests": n, "seconds": dt}
    O.set_threads(1)
    best = max(out.values(), key=lambda v: v["value"])
    return {"value": best["value"], "unit": UNIT, "cores": best["cores"], "kind": "oracle",
            "sample": f"first FCFS requests of the workload against its {len(sc.plans)} known plans, FP64 C "
                      f"oracle: {out['single']['requests']} in {out['single']['seconds']:.1f} s on one thread, "
                      f"{out['multi']['requests']} in {out['multi']['seconds']:.1f} s on {out['multi']['cores']} "
                      f"threads (host nproc {os.cpu_count()})",
            "single_thread": out["single"], "all_cores": out["multi"]}


def run_reference(args, sc):
    rank, _, world = dist_env()
    if rank != 0:
        return
    from oracle import Oracle

    per_step = max(1, args.ref_requests)
    times = []
    for i in range(args.warmup + args.steps):
        o = Oracle.from_scenario(sc)
        t0 = time.perf_counter()
        for r in sc.requests[:per_step]:
            o.schedule(r)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = per_step * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(sc, per_step),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {per_step} FCFS requests per step against {len(sc.plans)} known plans"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(sc, n_req, mode="batched"):
    return {"workload": sc.name, "known_plans": len(sc.plans), "requests_per_step": n_req,
            "actions": len(sc.actions), "max_horizon": int(sc.requests["horizon"].max()),
            "airspace_km": [round((sc.box[3] - sc.box[0]) / 1000), round((sc.box[4] - sc.box[1]) / 1000),
                            round((sc.box[5] - sc.box[2]) / 1000, 1)],
            "mode": {"batched": "FCFS through pipelined speculative batches (one persistent rollout launch fed by "
                                "the host; results identical to sequential FCFS)",
                     "waves": "FCFS through speculative waves (results identical to sequential FCFS)",
                     "sequential": "FCFS one request at a time"}[mode],
            "l2": "plan table (3 x 4096 x S fp32 planes) larger than L2 and rewritten by the restore every step",
            "parallelism": "replicas"}


def pct(a, q):
    import numpy as np

    return float(np.percentile(np.asarray(a, dtype=np.float64), q)) if len(a) else None


def timed(stream, fn, k, barrier):
    import torch

    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = None
    for _ in range(k):
        out = fn()
    e1.record(stream)
    barrier()
    return e0.elapsed_time(e1), out


def mlp_flops_per_row():
    """Multiply-adds of one forward pass of the proposal network (128 -> 4 x 256 -> 25), x 2."""
    dims = (128, 256, 256, 256, 256, 25)
    return 2.0 * sum(a * b for a, b in zip(dims[:-1], dims[1:]))


def train_learned(s, train_reqs, epochs=12):
    """Trains the proposal network on FastMDP rollouts of other requests (nothing admitted)."""
    import torch

    s.restore()
    rows = s.learned_collect(train_reqs)
    s.learned_init(7)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = s.learned_train(epochs=epochs, batch=512, lr=2e-3, seed=8)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    s.learned_clear_rows()
    s.restore()
    return {"rows": rows, "epochs": epochs, "final_loss": float(losses[-1]), "seconds": train_s,
            "params": s.learned_get_params()}


def sweep_point(s, sc, reqs, n_plain, stream, barrier, mx, world, learned_params=None, profile=False):
    """One known-plan count: plans/s and per-request time to result (closed batch: every
    request submitted at the call's start) of batched (pipelined), waves, plain sequential and
    learned FCFS over the same requests (plain: the first n_plain)."""
    out = {"known_plans": len(sc.plans), "requests": len(reqs), "workload": sc.name}

    def closed(label, fn, n, reps=2):
        fn()
        best, res_times = None, None
        for _ in range(reps):
            ms, val = timed(stream, fn, 1, barrier)
            ms = mx(ms)
            if best is None or ms < best:
                best, res_times = ms, s.last_call_times()
        out[label] = {"value": world * n / (best / 1e3), "unit": UNIT, "ms": best,
                      "time_to_result_ms_p50": pct(res_times, 50), "time_to_result_ms_p99": pct(res_times, 99)}
        return val

    s.stage(reqs)
    st0 = s.stats()

    def batched():
        s.restore()
        return s.schedule_staged(True)

    adm = closed("batched", batched, len(reqs))
    st = s.stats()
    out["batched"]["admitted"] = adm
    out["batched"]["rollouts_per_request"] = (st["batch_rollouts"] - st0["batch_rollouts"]) / (3 * len(reqs))
    s.set_batch_mode(1)
    st0 = s.stats()
    closed("waves", batched, len(reqs))
    st = s.stats()
    out["waves"]["waves_per_call"] = (st["batch_waves"] - st0["batch_waves"]) / 3
    s.set_batch_mode(0)
    s.stage(reqs[:n_plain])

    def plain():
        s.restore()
        return s.schedule_staged(False)

    closed("plain", plain, n_plain, reps=1)
    out["plain"]["requests"] = n_plain
    if learned_params is not None:
        s.learned_set_params(learned_params)
        s.restore()
        rep, acc, sp_, sf_ = s.learned_evaluate(reqs)
        # C5's own rule: a valid proposal (captured, no conflict, no terrain: the judge with an
        # unbounded step allowance) whose cost is within 5 % of FastMDP's plan of the request
        s.restore()
        _, valid, sp_u, sf_u = s.learned_evaluate(reqs, slack=1e9)
        c5 = int(((valid != 0) & (sp_u <= 1.05 * sf_u)).sum())

        def learned():
            s.restore()
            return s.schedule_learned(reqs, points=False)

        res, lrep = closed("learned", learned, len(reqs), reps=1)
        out["learned"].update({
            "accepted": int(lrep["accepted"]), "acceptance_rate": lrep["accepted"] / max(len(reqs), 1),
            "admitted": sum(r["verdict"] == 0 for r in res),
            "mean_cost_gap_vs_fastmdp": rep["mean_gap"], "max_cost_gap_vs_fastmdp": rep["max_gap"],
            "proposals_reaching_goal": rep["proposals_captured"], "proposal_steps": rep["proposal_steps"],
            "proposal_rollout_ms": rep["proposal_ms"], "fastmdp_rollout_ms": rep["fastmdp_ms"],
            "fastmdp_steps": rep["fastmdp_steps"],
            "judge": "reaches the goal, no conflict or terrain, steps <= 1.05 x fewest possible (gap <= 5 %)",
            "valid_proposals": int((valid != 0).sum()),
            "accepted_by_gap_to_fastmdp": c5, "acceptance_rate_by_gap_to_fastmdp": c5 / max(len(reqs), 1),
            "gap_rule": "valid proposal with steps <= 1.05 x FastMDP's steps for the same request"})
    s.restore()
    return out


def run_case(case):
    """Small cases for ncu captures: 20k known plans (C2's airspace), 64 requests."""
    import numpy as np
    import torch

    from paper_2008_03518_gb300 import scenarios as S
    from paper_2008_03518_gb300.fmdp import Scheduler

    sc = S.c3_batched(n_requests=64)
    with Scheduler.from_scenario(sc) as s:
        if case == "policy20k":
            s.learned_collect(S.make_requests(np.random.default_rng(2021), sc.box, 32, hm=sc.heightmap,
                                              zspan=(60.0, 500.0), tlo=0, thi=1800, horizon_range=(60, 1800),
                                              reach_frac=0.8, id0=10 ** 6))
            s.learned_init(7)
            s.learned_train(epochs=2, batch=512, lr=2e-3, seed=8)
            rep, acc, sp, sf = s.learned_evaluate(sc.requests)
            out = {"case": case, "proposal_steps": int(rep["proposal_steps"]), "proposal_ms": rep["proposal_ms"]}
        else:
            s.set_profiling(1)
            s.schedule_batch(sc.requests, points=False)
            st = s.stats()
            out = {"case": case, "sepcheck_launches": st["sepcheck_launches"], "sepcheck_ms": st["sepcheck_ms"]}
        torch.cuda.synchronize()
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fmdp", choices=["fmdp", "reference"])
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--ref-requests", type=int, default=6)
    ap.add_argument("--cpu-seconds", type=float, default=8.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-modes", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="arrival window per serving rate")
    ap.add_argument("--modes", default="sweep,learned,serving,departures,lookahead,cosim",
                    help="comma-separated extra modes to run")
    ap.add_argument("--time-scale", type=float, default=60.0, help="simulated seconds per wall second (serving)")
    ap.add_argument("--batch-mode", type=int, default=0, choices=[0, 1],
                    help="0: pipelined batches (default); 1: speculative waves (the ncu launch list)")
    ap.add_argument("--mode", default="batched", choices=["batched", "sequential"],
                    help="path timed for value: batched FCFS (default) or one request at a time")
    ap.add_argument("--metrics-jsonl", default=None,
                    help="also append the result line to this file (one JSON line per run)")
    ap.add_argument("--case", default=None, choices=["policy20k", "sepcheck20k"],
                    help="a small profiling case instead of the benchmark (one JSON line): the policy kernel "
                         "or the row-major separation check at 20k known plans")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.case:
        run_case(args.case)
        return

    rank, local_rank, world = dist_env()
    if world > 1:
        os.environ["CUDA_VISIBLE_DEVICES"] = str(local_rank)

    from paper_2008_03518_gb300 import scenarios as S

    sc = S.c2_plain_scale(n_requests=args.requests)
    if args.impl == "reference":
        run_reference(args, sc)
        return

    import numpy as np
    import torch

    reps = Replicas("nccl")  # one process per GPU; replicas exchange nothing but timings

    def barrier():
        reps.barrier()
        torch.cuda.synchronize()

    def mx(ms):
        return reps.max(ms)

    from paper_2008_03518_gb300.fmdp import Scheduler

    s = Scheduler.from_scenario(sc, batch_mode=args.batch_mode)
    stream = torch.cuda.current_stream()
    s.set_stream(stream.cuda_stream)
    s.snapshot()
    s.stage(sc.requests)
    n_req = len(sc.requests)
    tune = None
    if args.mode == "batched" and not args.no_tune:
        # launch shape of the batched rollout, tuned on the first batch (untimed set-up)
        tune = s.autotune(sc.requests[:256])

    def step(batched=args.mode == "batched"):
        s.restore()
        return s.schedule_staged(batched)

    for _ in range(args.warmup):
        step()
    s.set_profiling(0)  # resets the counters
    clocks = ClockSampler(local_rank if world == 1 else 0)
    clocks.start()
    ms, admitted = timed(stream, step, args.steps, barrier)
    clk = clocks.stop()
    st = s.stats()
    ms = mx(ms)
    value = world * n_req * args.steps / (ms / 1e3)
    times = s.last_call_times()
    gpu_launches = st["kernel_launches"]
    K = args.steps
    batch_stats = {"rollouts_per_step": st["batch_rollouts"] / K, "replans_per_step": st["batch_replans"] / K,
                   "resumed_replans_per_step": st["pipe_resumes"] / K,
                   "rechecks_per_step": st["pipe_rechecks"] / K,
                   "waves_per_step": st["batch_waves"] / K, "index_rebuild_drains_per_step": st["pipe_drains"] / K,
                   "persistent_ctas": st["pipe_ctas"], "resident_cta_slots": st["pipe_resident"],
                   "rollout_cta_occupancy": (st["pipe_cta_s"] / st["pipe_slot_s"]) if st["pipe_slot_s"] else None,
                   "rollout_occupancy_of_resident_slots":
                       (st["pipe_cta_s"] / (st["pipe_slot_s"] / max(st["pipe_ctas"], 1) * st["pipe_resident"]))
                       if st["pipe_slot_s"] else None,
                   "time_to_result_ms_p50": pct(times, 50), "time_to_result_ms_p99": pct(times, 99)}

    # ---- roofline of the rollout kernel and q_eval: one more step, profiled with CUDA events
    peaks_dev = s.probe_peaks()
    s.set_profiling(1)
    step()
    kt = s.stats()
    s.set_profiling(0)
    peaks, peak_kind = measured_peaks()
    launches = max(kt["rollout_launches"], 1)
    avg_ms = kt["rollout_ms"] / launches
    # algorithmic bytes: the 32-byte index items the steps read (the plan samples near the state)
    indexed = kt["items_scanned"] > 0
    bytes_per_launch = (32.0 * kt["items_scanned"] if indexed else 12.0 * kt["slots_scanned"]) / launches
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    tr = traffic_from_profile(os.path.join(ROOT, "paper_2008_03518_gb300", "csrc", "rollout.cu"))
    kernel_ms = {k: kt[k] for k in ("rollout_ms", "sepcheck_ms", "admit_ms", "influence_ms")}
    roofline = {"kernel": "rollout_kernel", "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "traffic": (tr * bytes_per_launch) if tr is not None else None,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_ms,
                "launches_per_step": launches, "threads_per_cta": kt["threads_per_cta"],
                "rollout_steps_per_step": kt["rollout_steps"], "indexed": indexed,
                "plan_samples_per_rollout_step": (kt["items_scanned"] if indexed else kt["slots_scanned"])
                / max(kt["rollout_steps"], 1),
                "launch": "pipelined: one persistent launch per step, timed with CUDA events on its stream"
                if args.batch_mode == 0 else "waves", "kernel_ms_per_step": kernel_ms}
    try:  # a secondary figure: never let it cost the bench line
        qe = q_eval_counted(kt, len(sc.actions), 5, peaks_dev, clk["sm_mhz"] if clk else None, kt["rollout_ms"])
    except Exception as e:  # noqa: BLE001
        qe = {"error": str(e)}

    modes = {} if not args.no_modes else None
    want = set(args.modes.split(",")) if not args.no_modes else set()
    learned3k = learned20k = None
    mlp = None
    if "learned" in want:
        tr3 = train_learned(s, S.make_requests(np.random.default_rng(2020), sc.box, 400, hm=sc.heightmap,
                                               zspan=(60.0, 500.0), tlo=0, thi=1800, horizon=1800, id0=10 ** 6))
        learned3k = tr3.pop("params")
        rows, ep, tsec = tr3["rows"], tr3["epochs"], tr3["seconds"]
        # a training row-epoch: forward, then gradients of the inputs and of the weights
        train_tflops = 3.0 * mlp_flops_per_row() * rows * ep / tsec / 1e12
        mlp = {"kernel": "MLP training (bf16 mma.sync GEMM, 64 x 64 tiles) and policy rollouts", "bound": "tensor",
               "training": {"achieved": train_tflops, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                            "frac": train_tflops / peaks["bf16_tflops"], "rows": rows, "epochs": ep,
                            "seconds": tsec, "final_loss": tr3["final_loss"]},
               "peak_source": f"{peak_kind} (MEASURED_PEAKS.json bf16_tflops, burst)"}
    if "sweep" in want:
        sweep = {"3k": sweep_point(s, sc, sc.requests, n_req, stream, barrier, mx, world, learned3k)}
        if mlp and "learned" in sweep["3k"]:
            L = sweep["3k"]["learned"]
            pol = L["proposal_steps"] * mlp_flops_per_row() / (L["proposal_rollout_ms"] / 1e3) / 1e12
            mlp["policy"] = {"achieved": pol, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                             "frac": pol / peaks["bf16_tflops"], "rows_stepped": L["proposal_steps"],
                             "ms": L["proposal_rollout_ms"]}
        sc3 = S.c3_batched(n_requests=512)
        s3 = Scheduler.from_scenario(sc3)
        s3.set_stream(stream.cuda_stream)
        s3.snapshot()
        if not args.no_tune:
            s3.autotune(sc3.requests[:256])
        if "learned" in want:
            tr20 = train_learned(s3, S.make_requests(np.random.default_rng(2021), sc3.box, 256, hm=sc3.heightmap,
                                                     zspan=(60.0, 500.0), tlo=0, thi=1800,
                                                     horizon_range=(60, 1800), reach_frac=0.8, id0=10 ** 6))
            learned20k = tr20.pop("params")
        sweep["20k"] = sweep_point(s3, sc3, sc3.requests, 128, stream, barrier, mx, world, learned20k)
        # the separation check of a pipelined call (exact report pass, row-major) at 20k plans
        s3.stage(sc3.requests)
        s3.set_profiling(1)
        s3.restore()
        s3.schedule_staged(True)
        k3 = s3.stats()
        s3.set_profiling(0)
        res3 = s3.fetch_staged()
        items = sum(len(p.xyz) for p in sc3.plans) + sum(r["n_points"] for r in res3 if r["verdict"] == 0)
        samples = sum(r["n_points"] for r in res3)
        # (request sample, plan sample of the same step) pairs the check measures
        per_row = np.zeros(sc3.n_slices_window + 1)
        for t0_, n_ in [(p.t0, len(p.xyz)) for p in sc3.plans] + \
                [(int(q["depart"]), r["n_points"]) for q, r in zip(sc3.requests, res3) if r["verdict"] == 0]:
            per_row[t0_] += 1
            per_row[t0_ + n_] -= 1
        cum = np.concatenate([[0.0], np.cumsum(np.cumsum(per_row))])
        pairs = float(sum(cum[int(q["depart"]) + r["n_points"]] - cum[int(q["depart"])]
                          for q, r in zip(sc3.requests, res3)))
        if k3["sepcheck_launches"] > 0 and k3["sepcheck_ms"] > 0:
            per = k3["sepcheck_ms"] / k3["sepcheck_launches"]
            b = 16.0 * items + 16.0 * samples
            fl = 10.0 * pairs / (per / 1e3) / 1e12
            sweep["sepcheck_rows_20k"] = {
                "kernel": "sepcheck_rows_kernel", "bound": "alu",
                "hbm": {"achieved": b / (per / 1e3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": b / (per / 1e3) / 1e9 / peaks["hbm_gbs"], "algorithmic_bytes_per_launch": b,
                        "bytes_from": "16 B per plan sample of every row (each row's items streamed once per "
                                      "launch) + 16 B per request sample"},
                "fp32": {"achieved": fl, "peak": peaks_dev["fp32_tflops"], "unit": "TFLOP/s",
                         "frac": fl / peaks_dev["fp32_tflops"], "pairs_per_launch": pairs,
                         "ops_from": "10 FP32 operations per (request sample, plan sample) pair: offsets, squared "
                                     "horizontal distance, |dz|, two threshold tests, two minima"},
                "avg_launch_ms": per, "launches": k3["sepcheck_launches"]}
        s3.close()
        sc4 = S.c4_serving()
        s4 = Scheduler.from_scenario(sc4)
        s4.set_stream(stream.cuda_stream)
        s4.snapshot()
        if not args.no_tune:
            s4.autotune(S.sweep_requests(sc4, 256, 7))
        sweep["100k"] = sweep_point(s4, sc4, S.sweep_requests(sc4, 512, 7), 128, stream, barrier, mx, world,
                                    learned20k)
        modes["sweep"] = sweep
        if "serving" in want:
            # serving at the 100k-plan table: Poisson arrivals, continuous batching, up to
            # saturation; each result equals one-at-a-time FCFS
            serving = {}
            sim0 = sc4.meta["sim_start"]
            rates = (50, 200, 1000, 2000, 4000, 8000, 16000, 32000, 64000, 128000)

            def window_s(rate):  # arrival window per offered rate (about 16k to 64k requests above 8k/s)
                return args.serve_seconds if rate <= 8000 else (1.0 if rate <= 32000 else 0.5)

            def serve_rate(rate):
                arr = S.poisson_arrivals(900 + rate, float(rate), window_s(rate))
                rq = S.serving_requests(sc4, arr, 901 + rate, time_scale=args.time_scale, sim_start=sim0)
                s4.restore()
                barrier()
                _, lat, rep = s4.serve(rq, arr, time_scale=args.time_scale, max_in_flight=256,
                                       max_active_plans=sc4.meta["max_active_plans"], sim_start_step=sim0,
                                       points=False)
                return {"requests": len(rq), "throughput_rps": rep["throughput_rps"],
                        "latency_p50_ms": rep["latency_p50_ms"],
                        "latency_p99_ms": rep["latency_p99_ms"], "latency_max_ms": rep["latency_max_ms"],
                        "admitted": rep["admitted"], "rollouts": rep["rollouts"],
                        "replans": rep["replans"], "max_in_flight_seen": rep["max_in_flight_seen"],
                        "expiries": rep["expiries"], "plans_expired": rep["plans_expired"],
                        "deferred_for_memory": rep["deferred_for_memory"],
                        "rollout_occupancy": rep["rollout_occupancy"], "drains": rep["drains"]}

            for rate in rates:
                serving[str(rate)] = serve_rate(rate)
            base = serving["50"]["latency_p99_ms"]

            def saturated(r, v):
                return v["throughput_rps"] < 0.9 * float(r) or v["latency_p99_ms"] > 10.0 * max(base, 1.0)

            knee = None
            for r in map(str, rates):
                if saturated(r, serving[r]):
                    # a rate that trips the rule runs once more: saturation shows in both runs,
                    # a passing stall of the host or the device in one (both are reported)
                    serving[r]["rerun"] = serve_rate(int(r))
                    if saturated(r, serving[r]["rerun"]):
                        knee = r
                        break
            modes["serving"] = {"known_plans": len(sc4.plans), "max_active_plans": sc4.meta["max_active_plans"],
                                "workload": sc4.name,
                                "arrivals": f"Poisson, {args.serve_seconds} s per rate (1 s for 16k-32k /s, 0.5 s above)",
                                "time_scale": args.time_scale, "sim_start_step": sim0, "rates_per_s": serving,
                                "saturation_rate": knee,
                                "saturation_rule": "first offered rate served below 0.9 x its rate or with p99 "
                                                   "above 10 x the p99 at 50 requests/s, in its run and in a "
                                                   "second run of the same arrivals"}
        s4.close()
    if mlp:
        modes["mlp_bf16"] = mlp
    if "departures" in want:
        # departure-time candidates: each request's eight variants (0 .. 7 minutes later)
        # planned together, the first admissible one admitted; requests in FCFS order
        delays = [60 * k for k in range(8)]
        nd = min(n_req, 128)

        def dep_step(batched):
            s.restore()
            _, ch, _ = s.schedule_departures(sc.requests[:nd], delays, points=False, batched=batched)
            return ch

        dep_step(True)
        mdep, ch = timed(stream, lambda: dep_step(True), 1, barrier)
        mdep = mx(mdep)
        mseq, ch_seq = timed(stream, lambda: dep_step(False), 1, barrier)
        mseq = mx(mseq)
        assert (ch_seq == ch).all(), "batched departures differ from one request at a time"
        modes["departures"] = {"known_plans": len(sc.plans), "value": world * nd / (mdep / 1e3), "unit": UNIT,
                               "ms_per_step": mdep, "requests_per_step": nd, "delays_s": delays,
                               "admitted": int((ch >= 0).sum()), "delayed": int((ch > 0).sum()),
                               "one_request_at_a_time": world * nd / (mseq / 1e3)}
    if "cosim" in want:
        nc = min(n_req, 128)

        def cs_step():
            s.restore()
            return s.schedule_cosim(sc.requests[:nc], points=False)

        cs_step()
        mcs, rcs = timed(stream, cs_step, 1, barrier)
        mcs = mx(mcs)
        modes["cosim"] = {"known_plans": len(sc.plans), "value": world * nc / (mcs / 1e3), "unit": UNIT,
                          "ms_per_step": mcs, "requests_per_step": nc,
                          "admitted": int(sum(r["verdict"] == 0 for r in rcs)),
                          "mode": "one cooperative launch, one CTA per request, grid barrier per step"}
    if "lookahead" in want:
        sce = S.e1_fine(n_requests=48)
        se = Scheduler.from_scenario(sce, lookahead_W=sce.meta["lookahead_W"])
        se.set_stream(stream.cuda_stream)
        se.snapshot()
        se.set_profiling(1)
        ref = se.schedule_many(sce.requests, points=False)
        steps_e = se.stats()["rollout_steps"]
        se.set_profiling(0)

        def la_step(batched):
            se.restore()
            if batched:
                return se.schedule_batch(sce.requests, points=False)
            return se.schedule_many(sce.requests, points=False)

        la_step(True)
        mla, got = timed(stream, lambda: la_step(True), 1, barrier)
        mla = mx(mla)
        mseq, _ = timed(stream, lambda: la_step(False), 1, barrier)
        mseq = mx(mseq)
        assert [r["verdict"] for r in got] == [r["verdict"] for r in ref], "batched lookahead differs"
        modes["lookahead_w10_dt01"] = {"known_plans": len(sce.plans), "value": world * len(sce.requests) / (mla / 1e3),
                                       "unit": UNIT, "ms_per_step": mla, "requests_per_step": len(sce.requests),
                                       "one_request_at_a_time": world * len(sce.requests) / (mseq / 1e3),
                                       "rollout_steps_one_at_a_time": steps_e,
                                       "us_per_rollout_step_one_at_a_time": 1e3 * mseq / max(steps_e, 1),
                                       "workload": sce.name}
        se.close()

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        # the known plans in pinned host memory, packed as the C ABI takes them
        def pinned(a):
            t = torch.empty(a.shape, dtype={np.float32: torch.float32, np.int32: torch.int32,
                                            np.int64: torch.int64}[a.dtype.type]).pin_memory()
            t.numpy()[...] = a
            return t

        pin = [pinned(np.array([p.t0 for p in sc.plans], dtype=np.int64)),
               pinned(np.array([len(p.xyz) for p in sc.plans], dtype=np.int32)),
               pinned(np.concatenate([np.asarray(p.xyz, dtype=np.float32) for p in sc.plans]))]
        t0s, counts, xyz = (t.numpy() for t in pin)
        h2d = t0s.nbytes + counts.nbytes + xyz.nbytes + n_req * 80

        def e2e_step():
            s.clear()
            s.add_plans_packed(t0s, counts, xyz)
            res = s.schedule_batch(sc.requests)
            return sum(r["xyz"].nbytes + r["actions"].nbytes + 48 for r in res)

        e2e_step()
        k = max(1, min(args.steps, 3))
        ems, d2h = timed(stream, e2e_step, k, barrier)
        ems = mx(ems)
        e2e = {"value": world * n_req * k / (ems / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": k,
               "api": "fmdp_clear + fmdp_add_plans (packed, pinned host arrays) + fmdp_schedule_batch"}

    p99 = None
    if modes and "serving" in modes:
        p99 = {r: v["latency_p99_ms"] for r, v in modes["serving"]["rates_per_s"].items()}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(sc, n_req, args.mode if args.batch_mode == 0 or args.mode != "batched"
                                      else "waves"),
            "admitted_per_step": admitted, "batch": batch_stats, "modes": modes, "e2e": e2e,
            "gpu_launches": gpu_launches, "roofline": roofline, "q_eval": qe, "device_peaks": peaks_dev,
            "clocks": clk, "p99_latency_ms_by_rate": p99, "autotune": tune}
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(sc, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
        if args.metrics_jsonl:
            from paper_2008_03518_gb300.fmdp import append_jsonl
            append_jsonl(args.metrics_jsonl, line)
    s.close()
    reps.close()


if __name__ == "__main__":
    main()
