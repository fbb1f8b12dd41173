"""Benchmark: FCFS flight-plan scheduling throughput (scheduled plans/s) on GB300.

Workload (default): the 30 km x 30 km x 1 km airspace with a 512^2 fractal heightmap,
3000 seeded multi-leg known plans and 1000 FCFS requests with 25 actions and horizons up
to 1800 steps. One step = one whole FCFS pass: the plan table is restored to the 3000
known plans (device copy) and the 1000 requests are planned, checked and admitted in
arrival order on the GPU, through speculative batches of 256 whose results are identical
to planning them one after the other. value = requests planned per second (admitted +
rejected).

  value    : requests already resident in device memory, trajectories left on the device
  modes    : the same workload planned one request at a time (plain sequential FCFS), and
             the 20k-known-plan workload (batches of 256, horizons U[60,1800]) batched
  e2e      : through the C ABI with host buffers: known plans uploaded from host memory,
             requests uploaded, trajectories and verdicts copied back, every step
  roofline : the rollout kernel (dominant), CUDA-event durations of a profiled step
  cpu_baseline: the FP64 oracle on this host's cores on a bounded sample

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


def q_eval_alu(kt, n_actions, n_wells, sm_max_mhz, n_sm=152, fp32_lanes=128):
    """q_eval (the well scan of the rollout) against the FP32 issue peak. Every plan sample a
    rollout step reads is tested against each well for each action: the well centre offset
    and the squared distance are 6 FMA (12 FP32 flops) per test. Peak: SMs x FP32 lanes per
    SM x 2 flops per FMA x the maximum SM clock."""
    steps, ms = kt.get("rollout_steps", 0), kt.get("rollout_ms", 0.0)
    samples = kt.get("items_scanned", 0) or kt.get("slots_scanned", 0)
    if steps <= 0 or ms <= 0.0 or samples <= 0:
        return None
    tests = float(samples) * n_actions * n_wells
    achieved = 12.0 * tests / (ms / 1e3) / 1e12
    peak = n_sm * fp32_lanes * 2.0 * sm_max_mhz * 1e6 / 1e12
    return {"kernel": "rollout_kernel (q_eval: the well scan)", "bound": "alu", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "flops_per_well_test": 12,
            "well_tests_per_rollout_step": tests / steps,
            "peak_from": f"{n_sm} SMs x {fp32_lanes} FP32 lanes x 2 flops x {sm_max_mhz:.0f} MHz"}


def cpu_baseline(sc, seconds=12.0):
    """The FP64 oracle, as it stands, on the first requests of the same workload."""
    from oracle import Oracle

    o = Oracle.from_scenario(sc)
    n = 0
    t0 = time.perf_counter()
    while n < len(sc.requests) and (time.perf_counter() - t0) < seconds:
        o.schedule(sc.requests[n])
        n += 1
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n} FCFS requests of the workload against its {len(sc.plans)} known plans, "
                      f"FP64 C oracle, one thread, {dt:.1f} s"}


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
            "mode": ("FCFS through speculative batches of 256 (results identical to sequential FCFS)"
                     if mode == "batched" else "FCFS one request at a time"),
            "l2": "plan table (3 x 4096 x S fp32 planes) larger than L2 and rewritten by the restore every step",
            "parallelism": "replicas"}


def learned_mode(S, s, sc, stream, barrier, max_over_ranks, world, train_requests):
    """The learned proposal on a workload: trained on FastMDP rollouts of other requests
    against the known plans, then evaluated (acceptance, cost gap against FastMDP) and
    timed as learned FCFS (accepted proposal, else FastMDP) over the workload's requests."""
    import numpy as np

    s.restore()
    t0 = time.perf_counter()
    rows = s.learned_collect(train_requests(np.random.default_rng(2020)))
    s.learned_init(7)
    losses = s.learned_train(epochs=12, batch=512, lr=2e-3, seed=8)
    train_s = time.perf_counter() - t0
    s.learned_clear_rows()
    s.restore()
    rep, acc, sp, sf = s.learned_evaluate(sc.requests)
    s.restore()
    s.schedule_learned(sc.requests, points=False)  # warm-up
    s.restore()
    ms, (res, lrep) = timed(stream, lambda: s.schedule_learned(sc.requests, points=False), 1, barrier)
    ms = max_over_ranks(ms)
    s.restore()
    n = len(sc.requests)
    return {"known_plans": len(sc.plans), "value": world * n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "requests": n, "accepted": int(lrep["accepted"]), "acceptance_rate": lrep["accepted"] / max(n, 1),
            "admitted": sum(r["verdict"] == 0 for r in res),
            "evaluate": {"accepted": rep["accepted"], "proposals_reaching_goal": rep["proposals_captured"],
                         "fastmdp_reaching_goal": rep["fastmdp_captured"], "mean_cost_gap": rep["mean_gap"],
                         "max_cost_gap": rep["max_gap"], "proposal_rollout_ms": rep["proposal_ms"],
                         "fastmdp_rollout_ms": rep["fastmdp_ms"],
                         "proposal_steps": rep["proposal_steps"], "fastmdp_steps": rep["fastmdp_steps"]},
            "training": {"rows": rows, "epochs": 12, "final_loss": float(losses[-1]), "seconds": train_s,
                         "requests": "400 (3k) / 256 (20k) other seeded requests, FastMDP rollouts"},
            "judge": "reaches the goal, no conflict or terrain, steps <= 1.05 x fewest possible (gap <= 5 %)"}


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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fmdp", choices=["fmdp", "reference"])
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--ref-requests", type=int, default=6)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-modes", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="batched mode: skip the launch-shape autotuner")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="arrival window per serving rate")
    ap.add_argument("--modes", default="sequential,departures,lookahead,cosim,learned,batched20k,learned20k,serving",
                    help="comma-separated extra modes to run")
    ap.add_argument("--time-scale", type=float, default=60.0, help="simulated seconds per wall second (serving)")
    ap.add_argument("--mode", default="batched", choices=["batched", "sequential"],
                    help="path timed for value: speculative batches (default) or one request at a time")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

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

    def max_over_ranks(ms):
        return reps.max(ms)

    from paper_2008_03518_gb300.fmdp import Scheduler

    s = Scheduler.from_scenario(sc)
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
    ms = max_over_ranks(ms)
    value = world * n_req * args.steps / (ms / 1e3)
    gpu_launches = st["kernel_launches"]
    batch_stats = {"waves_per_step": st["batch_waves"] / args.steps,
                   "rollouts_per_step": st["batch_rollouts"] / args.steps,
                   "replans_per_step": st["batch_replans"] / args.steps}

    # ---- roofline of the rollout kernel: one more step, launched eagerly with CUDA events
    s.set_profiling(1)
    step()
    kt = s.stats()
    s.set_profiling(0)
    peaks, peak_kind = measured_peaks()
    launches = max(kt["rollout_launches"], 1)
    avg_ms = kt["rollout_ms"] / launches
    # algorithmic bytes: the plan samples the steps must read (32-byte index items near the
    # state with the spatial index; 12-byte table samples of every slot without it)
    indexed = kt["items_scanned"] > 0
    bytes_per_launch = (32.0 * kt["items_scanned"] if indexed else 12.0 * kt["slots_scanned"]) / launches
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    tr = traffic_from_profile(os.path.join(ROOT, "paper_2008_03518_gb300", "csrc", "rollout.cu"))
    kernel_ms = {k: kt[k] for k in ("rollout_ms", "sepcheck_ms", "admit_ms", "influence_ms")}
    roofline = {"kernel": "rollout_kernel", "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "traffic": (tr * bytes_per_launch) if tr is not None else None,
                "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_ms,
                "launches_per_step": launches, "cluster_size": kt["cluster_size"],
                "threads_per_cta": kt["threads_per_cta"], "slots_per_cta": kt["slots_per_cta"],
                "rollout_steps_per_step": kt["rollout_steps"], "indexed": indexed,
                "plan_samples_per_rollout_step": (kt["items_scanned"] if indexed else kt["slots_scanned"])
                / max(kt["rollout_steps"], 1),
                "share_of_kernel_time": kt["rollout_ms"] / max(sum(kernel_ms.values()), 1e-9),
                "kernel_ms_per_step": kernel_ms}
    try:  # a secondary figure: never let it cost the bench line
        n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        qalu = q_eval_alu(kt, len(sc.actions), 5, float(peaks.get("sm_max_mhz", 2070.0)), n_sm=n_sm)
        if qalu and clk and clk.get("sm_mhz"):  # the same work against the clock the run saw
            qalu["frac_at_median_clock"] = qalu["frac"] * float(peaks.get("sm_max_mhz", 2070.0)) / clk["sm_mhz"]
            qalu["median_sm_mhz"] = clk["sm_mhz"]
    except Exception as e:  # noqa: BLE001
        qalu = {"error": str(e)}

    # ---- other modes of the metric: plain sequential FCFS, and 20k known plans batched
    modes = None
    want = set(args.modes.split(",")) if not args.no_modes else set()
    if want:
        modes = {}
    if "sequential" in want:
        step(False)
        mseq, _ = timed(stream, lambda: step(False), 1, barrier)
        mseq = max_over_ranks(mseq)
        modes["plain_sequential"] = {"known_plans": len(sc.plans), "value": world * n_req / (mseq / 1e3),
                                     "unit": UNIT, "ms_per_step": mseq,
                                     "mode": "one request at a time, each rollout one cluster launch"}
    if want:
        modes["batched"] = {"known_plans": len(sc.plans), "value": value, "unit": UNIT}
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
        mdep = max_over_ranks(mdep)
        mseq, ch_seq = timed(stream, lambda: dep_step(False), 1, barrier)
        mseq = max_over_ranks(mseq)
        assert (ch_seq == ch).all(), "batched departures differ from one request at a time"
        modes["departures"] = {"known_plans": len(sc.plans), "value": world * nd / (mdep / 1e3), "unit": UNIT,
                               "ms_per_step": mdep, "requests_per_step": nd, "delays_s": delays,
                               "admitted": int((ch >= 0).sum()), "delayed": int((ch > 0).sum()),
                               "one_request_at_a_time": world * nd / (mseq / 1e3),
                               "mode": "each request's 8 departure variants; the variants of 32 requests per "
                                       "speculative batch (results equal one request at a time, also timed), FCFS"}
    if "cosim" in want:
        # batch co-simulation: 128 requests of the workload stepping on one clock, each seeing
        # the others' wells, then admitted in array order
        nc = min(n_req, 128)

        def cs_step():
            s.restore()
            return s.schedule_cosim(sc.requests[:nc], points=False)

        cs_step()
        mcs, rcs = timed(stream, cs_step, 1, barrier)
        mcs = max_over_ranks(mcs)
        modes["cosim"] = {"known_plans": len(sc.plans), "value": world * nc / (mcs / 1e3), "unit": UNIT,
                          "ms_per_step": mcs, "requests_per_step": nc,
                          "admitted": int(sum(r["verdict"] == 0 for r in rcs)),
                          "mode": "one cooperative launch, one CTA per request, grid barrier per step"}
    if "lookahead" in want:
        # the paper's fidelity: W = 10 sub-steps of 0.1 s; 48 requests through speculative
        # waves of lookahead rollouts, and the same requests one at a time
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
        mla = max_over_ranks(mla)
        mseq, _ = timed(stream, lambda: la_step(False), 1, barrier)
        mseq = max_over_ranks(mseq)
        assert [r["verdict"] for r in got] == [r["verdict"] for r in ref], "batched lookahead differs"
        modes["lookahead_w10_dt01"] = {"known_plans": len(sce.plans), "value": world * len(sce.requests) / (mla / 1e3),
                                       "unit": UNIT, "ms_per_step": mla, "requests_per_step": len(sce.requests),
                                       "one_request_at_a_time": world * len(sce.requests) / (mseq / 1e3),
                                       "rollout_steps_one_at_a_time": steps_e,
                                       "us_per_rollout_step_one_at_a_time": 1e3 * mseq / max(steps_e, 1),
                                       "workload": sce.name}
        se.close()
    if "learned" in want:
        modes["learned"] = learned_mode(S, s, sc, stream, barrier, max_over_ranks, world,
                                        lambda rng: S.make_requests(rng, sc.box, 400, hm=sc.heightmap,
                                                                    zspan=(60.0, 500.0), tlo=0, thi=1800,
                                                                    horizon=1800, id0=10 ** 6))
    if "batched20k" in want or "learned20k" in want:
        sc3 = S.c3_batched(n_requests=512)
        s3 = Scheduler.from_scenario(sc3)
        s3.set_stream(stream.cuda_stream)
        s3.snapshot()
        s3.stage(sc3.requests)
        tune3 = None if args.no_tune else s3.autotune(sc3.requests[:256])

        def step3():
            s3.restore()
            return s3.schedule_staged(True)

        step3()
        s3.set_profiling(0)
        m3, adm3 = timed(stream, step3, 2, barrier)
        st3 = s3.stats()
        m3 = max_over_ranks(m3)
        if "learned20k" in want:
            modes["learned_20k"] = learned_mode(S, s3, sc3, stream, barrier, max_over_ranks, world,
                                                lambda rng: S.make_requests(rng, sc3.box, 256, hm=sc3.heightmap,
                                                                            zspan=(60.0, 500.0), tlo=0, thi=1800,
                                                                            horizon_range=(60, 1800),
                                                                            reach_frac=0.8, id0=10 ** 6))
        modes["batched_20k"] = {"known_plans": len(sc3.plans), "value": world * 512 * 2 / (m3 / 1e3),
                                "unit": UNIT, "ms_per_step": m3 / 2, "requests_per_step": 512,
                                "batch": 256, "admitted_per_step": adm3,
                                "waves_per_step": st3["batch_waves"] / 2,
                                "replans_per_step": st3["batch_replans"] / 2, "workload": sc3.name,
                                "autotune": tune3}
        s3.close()

    if "serving" in want:
        # serving: Poisson arrivals against a sliding-window table (60 km, 40k known plans,
        # room for 100k), continuous batching; each result equals one-at-a-time FCFS
        sc4 = S.c4_serving()
        s4 = Scheduler.from_scenario(sc4)
        s4.set_stream(stream.cuda_stream)
        s4.snapshot()
        serving = {}
        for rate in (50, 200, 1000, 2000):
            arr = S.poisson_arrivals(900 + rate, float(rate), args.serve_seconds)
            rq = S.serving_requests(sc4, arr, 901 + rate, time_scale=args.time_scale)
            s4.restore()
            barrier()
            _, lat, rep = s4.serve(rq, arr, time_scale=args.time_scale, max_in_flight=512, points=False)
            serving[str(rate)] = {"requests": len(rq), "throughput_rps": rep["throughput_rps"],
                                  "latency_p50_ms": rep["latency_p50_ms"], "latency_p99_ms": rep["latency_p99_ms"],
                                  "latency_max_ms": rep["latency_max_ms"], "admitted": rep["admitted"],
                                  "waves": rep["waves"], "replans": rep["replans"],
                                  "max_in_flight_seen": rep["max_in_flight_seen"], "expiries": rep["expiries"],
                                  "plans_expired": rep["plans_expired"]}
        modes["serving"] = {"known_plans": len(sc4.plans), "max_plans": sc4.max_slots, "workload": sc4.name,
                            "arrivals": f"Poisson, {args.serve_seconds} s per rate",
                            "time_scale": args.time_scale, "rates_per_s": serving}
        s4.close()

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
        d2h = 0

        def e2e_step():
            s.clear()
            s.add_plans_packed(t0s, counts, xyz)
            res = s.schedule_batch(sc.requests)
            return sum(r["xyz"].nbytes + r["actions"].nbytes + 48 for r in res)

        e2e_step()
        k = max(1, min(args.steps, 3))
        ems, d2h = timed(stream, e2e_step, k, barrier)
        ems = max_over_ranks(ems)
        e2e = {"value": world * n_req * k / (ems / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": k, "api": "fmdp_clear + fmdp_add_plans (packed, pinned host arrays) + fmdp_schedule_batch"}

    p99 = None
    if modes and "serving" in modes:
        p99 = {r: v["latency_p99_ms"] for r, v in modes["serving"]["rates_per_s"].items()}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(sc, n_req, args.mode),
            "admitted_per_step": admitted, "batch": batch_stats, "modes": modes, "e2e": e2e,
            "gpu_launches": gpu_launches, "roofline": roofline, "q_eval_alu": qalu, "clocks": clk,
            "p99_latency_ms_by_rate": p99, "autotune": tune}
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(sc, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    reps.close()


if __name__ == "__main__":
    main()
