"""Benchmark of the constrained-motion hot path on one GB300 (or N replicas).

Prints one JSON line: whole-job constrained waypoints/s (projection + FK + CC) of the CUDA
library on seeded synthetic workloads, with the dominant kernel's roofline, an end-to-end
figure through the C ABI with host buffers, and the FP64 oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload validate|plan]
  python bench.py --impl reference ...   # the oracle arm (CPU), same workload and metric
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2505_06791_gb300 import synth as S  # noqa: E402

METRIC = "constrained waypoints/s (proj+FK+CC); p50 plan ms, learned vs plain @1e-4 resid"
UNIT = "waypoints/s"

# ---- algorithmic work per unit (FP32 operations of the method as the kernels state it;
#      FMA = 2, add/mul/min/max/compare = 1, each sin/cos pair, atan2, sqrt, rsqrt and
#      divide = 1) ----
F_CHAIN_JOINT = 48          # one DH joint of the chain (u, v, p, y, z columns)
F_TASK_RP_JOINT = 8         # roll/pitch task-Jacobian entries per joint
F_TASK_RP_FIXED = 12        # Euler angles and the rate map (2 atan2, sqrt, rsqrt, div, ...)
F_DAMPED_JOINT = 9          # J J^T accumulation (6) + g = J^T y (3) per joint
F_DAMPED_FIXED = 10         # 2x2 solve
F_UPDATE_JOINT = 10         # smoothing hinge, update, clamp per joint
F_VALIDITY = 4
F_SPHERE_FK = 18            # R c + p
F_PAIR_SPHERE = 11
F_PAIR_BOX = 34
F_PAIR_CAPSULE = 25


def flops_waypoint_iter(dof: int) -> int:
    return (dof * (F_CHAIN_JOINT + F_TASK_RP_JOINT + F_DAMPED_JOINT + F_UPDATE_JOINT)
            + dof + F_TASK_RP_FIXED + F_DAMPED_FIXED + F_VALIDITY)


def flops_cc_waypoint(n_spheres: int, n_sph: int, n_box: int, n_cap: int) -> int:
    return n_spheres * (F_SPHERE_FK + n_sph * F_PAIR_SPHERE + n_box * F_PAIR_BOX
                        + n_cap * F_PAIR_CAPSULE)


def algorithmic_flops(dof, W, S_, scene_counts, status, first_fail, iters):
    """Work the method evaluates for these outcomes: Alg. 1 evaluates waypoints 1..W-1 in
    each of its iterations; FK + CC walk waypoints 0..first colliding one (all W if valid,
    none if the projection failed)."""
    status = np.asarray(status).astype(np.int64)
    ff = np.asarray(first_fail).astype(np.int64)
    it = np.asarray(iters).astype(np.int64)
    proj = (it * (W - 1)).sum() * flops_waypoint_iter(dof)
    cc_wp = np.where(status == 0, W, np.where(status == 2, ff + 1, 0)).sum()
    return float(proj + cc_wp * flops_cc_waypoint(S_, *scene_counts)), int(cc_wp)


def executed_flops(dof: int, counters) -> float:
    """FLOPs of the work the kernels evaluated (cprrtc_work_counters): Alg. 1 waypoint
    updates, DH chains of the collision check, points moved to world coordinates, and
    ball-vs-primitive tests by primitive."""
    upd, chains, tf, ps, pb, pc = [float(x) for x in counters[:6]]
    return (upd * flops_waypoint_iter(dof) + chains * dof * F_CHAIN_JOINT + tf * F_SPHERE_FK
            + ps * F_PAIR_SPHERE + pb * F_PAIR_BOX + pc * F_PAIR_CAPSULE)


def profiled_traffic_per_unit(name: str, key: str):
    """DRAM bytes per unit recorded in profiles/<name> from an ncu capture, or None when the
    kernel's sources (the files the profile lists) changed since (the file records their
    hash)."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", name)
    try:
        text = open(path).read()
    except OSError:
        return None
    m_hash = re.search(r"source_sha256_16: ([0-9a-f]{16})", text)
    m_files = re.search(r"source_files: ([\w. ]+)", text)
    m_val = re.search(key + r": ([0-9.eE+]+)", text)
    if not (m_hash and m_val and m_files):
        return None
    csrc = os.path.join(ROOT, "paper_2505_06791_gb300", "csrc")
    try:
        blob = b"".join(open(os.path.join(csrc, f), "rb").read() for f in sorted(m_files.group(1).split()))
    except OSError:
        return None
    h = hashlib.sha256(blob).hexdigest()[:16]
    return float(m_val.group(1)) if h == m_hash.group(1) else None


def fp32_peak_tflops(sm_count: int, mhz: float) -> float:
    """FP32 FMA-pipe peak: SMs x 128 lanes x 2 FLOP x clock."""
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


def fp32_peak(ctx, sm_count: int, peaks: dict):
    """(peak TFLOP/s, note) for the FP32-ALU rooflines: measured on this GPU by the library's
    FMA-chain kernel (after the timed region), with the nominal unit-count figure beside it;
    the nominal figure only if the measurement fails."""
    mhz = peaks.get("sm_max_mhz", 2070.0)
    nominal = fp32_peak_tflops(sm_count, mhz)
    try:
        measured = ctx.measure_fp32_peak()
    except Exception as exc:  # the roofline's denominator only; the step is already timed
        return nominal, (f"FP32 FMA pipe, nominal: {sm_count} SMs x 128 x 2 x {mhz:.0f} MHz "
                         f"(measurement failed: {exc})")
    return measured, (f"FP32 FMA measured on this GPU: scalar and packed FMA chains on every SM "
                      f"(cprrtc_measure_fp32_peak), {measured:.1f} TFLOP/s; nominal {sm_count} "
                      f"SMs x 128 x 2 x {mhz:.0f} MHz = {nominal:.1f}")


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for name, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# workloads

VAL_SWEEP = (256, 4096, 65536)


def validation_workload(seed=1):
    """7-DOF arm (59 spheres), 16 obstacle spheres in the 1.2 m cube, 256 motions x 32
    waypoints between uniform configurations, roll/pitch constraint, <= 20 iterations."""
    rb = S.make_arm7(seed)
    sc = S.make_scene(1000 + seed, n_sph=16)
    c = S.roll_pitch(20)
    return rb, sc, c, 256, 32


def manifold_starts_gpu(ctx, rb, n, seed):
    """Uniform configurations projected onto the manifold by the library (inputs only)."""
    import torch
    out = []
    k = 0
    while sum(len(o) for o in out) < n:
        q = torch.from_numpy(S.uniform_configs(rb, 2 * n, seed + k).astype(np.float32)).cuda()
        r = ctx.project_configs(q, 60)
        ok = r["ok"].bool()
        out.append(r["q"][ok])
        k += 1
    return torch.cat(out)[:n].contiguous()


PLAN_N = 1000
PLAN_PARAMS = dict(range_=0.3, W=32, max_rounds=1000, workers=8, max_nodes=2048,
                   max_connect=32, max_path=512)
# the planner's time-sliced schedule (cprrtc_set_plan_slicing): first slice, later slices (rounds)
PLAN_SLICING = (100, 50)


def planner_scenes(n, seed=2):
    """Full planner: per-problem scenes of 200 mixed obstacles (100 spheres, 60 oriented boxes,
    40 capsules) in a 3 x 3 x 1.8 m workspace around the arm, base keep-out 0.35 m."""
    return [S.make_planning_scene(2_000_000 + 10_007 * seed + p) for p in range(n)]


def gpu_start_goal(rb, c, scenes, seed, device):
    """Start/goal per problem: uniform configurations projected by the library, kept when
    collision-free with every robot sphere inflated by 1 mm (library collision check)."""
    import torch
    from paper_2505_06791_gb300.capi import Context
    proj = Context(device)
    proj.set_robot(rb)
    proj.set_constraint(c)
    inflated = S.Robot(rb.joints, rb.ee, rb.spheres.copy())
    inflated.spheres[:, 4] += 1e-3
    chk = Context(device)
    chk.set_robot(inflated)
    chk.set_constraint(S.no_constraint())
    starts, goals = [], []
    for p, sc in enumerate(scenes):
        chk.set_obstacles(sc)
        found = []
        k = 0
        while len(found) < 2:
            cand = torch.from_numpy(S.uniform_configs(rb, 64, seed * 1_000_003 + 977 * p + k)
                                    .astype(np.float32)).cuda()
            r = proj.project_configs(cand, 60)
            qp = r["q"][r["ok"].bool()].contiguous()
            if len(qp):
                v = chk.validate(qp, qp, 2, with_q=False)
                free = qp[v["status"] == 0]
                found += [free[i] for i in range(min(2 - len(found), len(free)))]
            k += 1
            if k > 200:
                raise RuntimeError(f"no collision-free start/goal for problem {p}")
        starts.append(found[0])
        goals.append(found[1])
    proj.close()
    chk.close()
    return torch.stack(starts).contiguous(), torch.stack(goals).contiguous()


def plan_flops(dof, scenes, n_spheres, work):
    work = np.asarray(work, dtype=np.float64)
    f_iter = flops_waypoint_iter(dof)
    f_cc = np.array([flops_cc_waypoint(n_spheres, len(sc.sph), len(sc.box), len(sc.cap))
                     for sc in scenes])
    return float((work[:, 0] * f_iter + work[:, 1] * f_cc).sum())


def run_plan(args, world, rank, local):
    import torch
    from paper_2505_06791_gb300 import build
    from paper_2505_06791_gb300.capi import Context
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rb, c = S.make_arm7(1), S.roll_pitch(20)
    n = args.problems
    # each rank plans its own seeded problems (weak scaling, no collective)
    seed = 2 + 1000 * rank
    scenes = planner_scenes(n, seed)
    start, goal = gpu_start_goal(rb, c, scenes, seed, local)
    stream = torch.cuda.Stream(device=dev)
    ctx = Context(local, stream.cuda_stream)
    ctx.set_robot(rb)
    ctx.set_constraint(c)
    ctx.set_scene_batch(scenes)
    ctx.set_plan_slicing(*PLAN_SLICING)
    prm = ctx.plan_params(seed=seed, **PLAN_PARAMS)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        out = ctx.alloc_plan_outputs(n, prm, start, edges=False)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        for _ in range(args.warmup):
            ctx.plan(start, goal, prm, out=out)
        stream.synchronize()
        ctx.set_timing(True)
        ctx.reset_timing()
        ctx.work_counters(reset=True)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        clocks = ClockSampler(local)
        barrier(world)
        torch.cuda.synchronize()
        clocks.start()
        for k in range(args.steps):
            flush.fill_(float(k))            # evict L2 between steps (write > L2 size)
            starts[k].record(stream)
            ctx.plan(start, goal, prm, out=out)
            ends[k].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        clk = clocks.stop()
        step_ms = [s_.elapsed_time(e) for s_, e in zip(starts, ends)]
        kms, launches = ctx.kernel_time("plan")
        counters = ctx.work_counters() / max(args.steps, 1)
        ctx.set_timing(False)
    total_ms = max_over_ranks(sum(step_ms), world)
    L = out["path_len"].cpu().numpy()
    wp = out["waypoints"].cpu().numpy()
    ms = out["plan_ms"].cpu().numpy()
    work = out["work"].cpu().numpy()
    rounds = out["rounds"].cpu().numpy()

    waypoints_step = int(wp.sum())
    value = sum_over_ranks(waypoints_step, world) * args.steps / (total_ms / 1e3)
    nominal = plan_flops(rb.dof, scenes, len(rb.spheres), work)

    # the same problems on one CTA per problem, each planned in one stretch (the schedule
    # without time slicing), timed alike: same search, so the same outputs
    schedule = None
    if args.schedule_ab:
        with torch.cuda.stream(stream):
            ctx.set_plan_slicing(0)
            out_f = ctx.alloc_plan_outputs(n, prm, start, edges=False)
            ctx.plan(start, goal, prm, out=out_f)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            barrier(world)
            torch.cuda.synchronize()
            for k in range(args.steps):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                ctx.plan(start, goal, prm, out=out_f)
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            barrier(world)
            f_ms = max_over_ranks(sum(x.elapsed_time(y) for x, y in ev), world)
            ctx.set_plan_slicing(*PLAN_SLICING)
        same = all(np.array_equal(out_f[k].cpu().numpy(), out[k].cpu().numpy())
                   for k in ("path_len", "rounds", "waypoints", "work"))
        msf = out_f["plan_ms"].cpu().numpy()
        sf = out_f["path_len"].cpu().numpy() > 0
        schedule = {
            "time_sliced": {"first_slice_rounds": PLAN_SLICING[0], "slice_rounds": PLAN_SLICING[1],
                            "ms_per_step": total_ms / args.steps,
                            "mean_problems_in_flight": float(ms.sum()) / (total_ms / args.steps)},
            "one_cta_per_problem": {"ms_per_step": f_ms / args.steps,
                                    "mean_problems_in_flight": float(msf.sum()) / (f_ms / args.steps),
                                    "p50_plan_ms": float(np.percentile(msf[sf], 50)) if sf.any() else None,
                                    "p95_plan_ms": float(np.percentile(msf[sf], 95)) if sf.any() else None},
            "speedup": f_ms / total_ms,
            "same_outputs": bool(same),
            "note": "persistent CTAs; an unsolved problem goes back to the queue's tail between "
                    "slices while others wait, so the long problems share the GPU to the end; "
                    "plan_ms is the device time of a problem's slices; problems in flight = the "
                    "sum of plan_ms over the step (the GPU holds 2 per SM at once)",
        }

    # the learned form on the same problems: the network trained first (untimed), every extend
    # motion warm-started by it, plain Alg. 1 as judge and fallback
    learned = None
    if args.learned:
        with torch.cuda.stream(stream):
            tr = train_warm_network(ctx, rb, 40 + 1000 * rank, dev, args.train_epochs, stream)
            ctx.set_plan_warm_start(WS_REFINE)
            out_w = ctx.alloc_plan_outputs(n, prm, start, edges=False)
            for _ in range(max(1, args.warmup)):
                ctx.plan(start, goal, prm, out=out_w)
            ctx.work_counters(reset=True)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            barrier(world)
            torch.cuda.synchronize()
            for k in range(args.steps):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                ctx.plan(start, goal, prm, out=out_w)
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            barrier(world)
            w_ms = max_over_ranks(sum(x.elapsed_time(y) for x, y in ev), world)
            wcnt = ctx.work_counters() / max(args.steps, 1)
            ctx.set_plan_warm_start(0)
        Lw = out_w["path_len"].cpu().numpy()
        msw = out_w["plan_ms"].cpu().numpy()
        sw = Lw > 0
        learned = {
            "ms_per_step": w_ms / args.steps,
            "value": sum_over_ranks(int(out_w["waypoints"].sum().item()), world) * args.steps / (w_ms / 1e3),
            "p50_plan_ms": float(np.percentile(msw[sw], 50)) if sw.any() else None,
            "p95_plan_ms": float(np.percentile(msw[sw], 95)) if sw.any() else None,
            "success_rate": float(sw.mean()),
            "mean_rounds": float(out_w["rounds"].cpu().numpy().mean()),
            "extend_motions_warm_started_per_step": float(wcnt[6]),
            "warm_segments_accepted_per_step": float(wcnt[7]),
            "network": {"train_pairs": WS_TRAIN, "epochs": args.train_epochs, "refine_iters": WS_REFINE,
                        "pairs_from": "cprrtc_project_configs (the tests train on oracle pairs)",
                        "held_out_loss": [float(tr["held0"]), float(tr["held1"])],
                        "zero_prediction_loss": tr["zero_loss"], "train_s": tr["train_s"]},
            "note": "extend motions warm-started by the network's correction of their end, spread "
                    "along the motion; Alg. 1 judges and falls back; connect steps unchanged",
        }
    flops = executed_flops(rb.dof, counters)

    # end to end through the C ABI with pinned host buffers
    h_start = start.cpu().pin_memory()
    h_goal = goal.cpu().pin_memory()
    h_out = {k: (torch.empty(v.shape, dtype=v.dtype).pin_memory() if v is not None else None)
             for k, v in out.items()}
    ctx.plan(h_start, h_goal, prm, out=h_out)
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        ctx.plan(h_start, h_goal, prm, out=h_out)
    e2e_s = time.perf_counter() - t0
    h2d = 2 * n * rb.dof * 4
    d2h = sum(v.numel() * v.element_size() for v in h_out.values() if v is not None)
    e2e = {"value": waypoints_step * e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    peaks = load_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak, peak_note = fp32_peak(ctx, sm_count, peaks)
    avg_kernel_s = kms / 1e3 / max(launches, 1)
    achieved = flops / avg_kernel_s / 1e12
    solved = L > 0
    per_round = profiled_traffic_per_unit("plan_kernel_planner_1000_problems.md",
                                          "traffic_per_problem_round_bytes")
    traffic = None if per_round is None else per_round * float(rounds.sum())
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "full planner, plain form: RRT-Connect on a 7-DOF arm among 200 mixed obstacles per problem, roll-pitch", "problems": n,
                   "dof": rb.dof, "robot_spheres": len(rb.spheres),
                   "obstacles_per_problem": {"spheres": 100, "boxes": 60, "capsules": 40},
                   "constraint": "roll-pitch", "range": PLAN_PARAMS["range_"],
                   "W": PLAN_PARAMS["W"], "max_rounds": PLAN_PARAMS["max_rounds"],
                   "workers_per_problem": PLAN_PARAMS["workers"],
                   "schedule": f"time-sliced persistent CTAs (first slice {PLAN_SLICING[0]} rounds, "
                               f"then {PLAN_SLICING[1]})",
                   "l2": "flushed (256 MB write) between steps",
                   "recipe_departure": "obstacle centres in a 3 x 3 x 1.8 m workspace with a 0.35 m "
                                       "keep-out around the base instead of the 1.2 m cube: with "
                                       "200 obstacles the cube leaves no collision-free configuration",
                   "parallelism": f"replicas x{world}"},
        "p50_plan_ms": float(np.percentile(ms[solved], 50)) if solved.any() else None,
        "p95_plan_ms": float(np.percentile(ms[solved], 95)) if solved.any() else None,
        "p50_plan_ms_all": float(np.percentile(ms, 50)),
        "success_rate": float(solved.mean()),
        "learned_vs_plain": {"plain": {"p50_plan_ms": float(np.percentile(ms[solved], 50)) if solved.any() else None,
                                       "p95_plan_ms": float(np.percentile(ms[solved], 95)) if solved.any() else None,
                                       "success_rate": float(solved.mean()),
                                       "ms_per_step": total_ms / args.steps},
                             "learned": learned},
        "waypoints_per_step": waypoints_step,
        "evaluated_waypoints_per_s": sum_over_ranks(int(work[:, 1].sum()), world) * args.steps
                                     / (total_ms / 1e3),
        "evaluated_note": "waypoints of attempted motions that went through projection, FK and "
                          "CC (motions that fail projection or collide early count only what "
                          "was checked); `value` counts W per attempted motion",
        "mean_rounds": float(rounds.mean()),
        "schedule": schedule,
        "e2e": e2e,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "plan_kernel",
                     "traffic_note": "ncu DRAM bytes per problem-round of a 304-problem capture "
                                     "(profiles/plan_kernel_planner_1000_problems.md) x problem-rounds",
                     "flop_per_launch": flops, "avg_launch_ms": avg_kernel_s * 1e3,
                     "work_per_launch": {"alg1_updates": float(counters[0]),
                                         "cc_chains": float(counters[1]),
                                         "transforms": float(counters[2]),
                                         "tests_sph_box_cap": [float(x) for x in counters[3:6]]},
                     "peak_note": peak_note},
        "all_pairs_equivalent": {"flop_per_launch": nominal,
                                 "tflops": nominal / avg_kernel_s / 1e12,
                                 "note": "FLOPs a check of every robot sphere against every "
                                         "obstacle would take for the same waypoints"},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    inputs = (rb, c, scenes, start.cpu().numpy(), goal.cpu().numpy(), seed)
    return line, inputs


def oracle_plan_sample(rb, c, scenes, start, goal, seed, budget_s, threads):
    """Oracle planner over the first problems of the workload, one problem per host thread,
    until the time budget is spent. Returns (waypoints/s, per-problem ms, #problems)."""
    import concurrent.futures as cf
    import oracle

    def one(p):
        orc = oracle.Oracle(rb, scenes[p], c)
        t = time.perf_counter()
        r = orc.plan(start[p:p + 1], goal[p:p + 1], range_=PLAN_PARAMS["range_"],
                     W=PLAN_PARAMS["W"], max_rounds=PLAN_PARAMS["max_rounds"],
                     n_workers=PLAN_PARAMS["workers"], max_nodes=PLAN_PARAMS["max_nodes"],
                     max_connect=PLAN_PARAMS["max_connect"], seed=seed,
                     max_path=PLAN_PARAMS["max_path"])
        return (time.perf_counter() - t) * 1e3, int(r["waypoints"][0]), int(r["path_len"][0] > 0)

    t0 = time.perf_counter()
    res = []
    p = 0
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        while p < len(scenes) and time.perf_counter() - t0 < budget_s:
            batch = list(range(p, min(p + threads, len(scenes))))
            res += list(ex.map(one, batch))
            p += len(batch)
    el = time.perf_counter() - t0
    wp = sum(r[1] for r in res)
    return wp / el, [r[0] for r in res], len(res), sum(r[2] for r in res), el


def cpu_baseline_plan(inputs, budget_s):
    rb, c, scenes, start, goal, seed = inputs
    cores = os.cpu_count() or 1
    v, ms, n, solved, el = oracle_plan_sample(rb, c, scenes, start, goal, seed, budget_s, cores)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {n} of the {len(scenes)} problems, one per thread ({el:.1f} s); "
                      f"solved {solved}, p50 plan {np.percentile(ms, 50):.0f} ms per problem"}


BATCH_N = 512
BATCH_PARAMS = dict(range_=0.3, max_rounds=1000, workers=8, max_nodes=2048, max_connect=32,
                    max_path=512)


def gpu_batch_start_goal(robots, cons, problems, scenes, seed, device):
    """Start/goal [n][8] per problem with the library: uniform configurations of the
    problem's robot, projected under its constraint, kept when collision-free with every
    robot sphere inflated by 1 mm."""
    import torch
    from paper_2505_06791_gb300.capi import Context
    proj, chk = Context(device), Context(device)
    start = torch.zeros((len(problems), 8), device="cuda")
    goal = torch.zeros((len(problems), 8), device="cuda")
    cur_r = None
    for p, (r, c, sc, W) in enumerate(problems):
        rb = robots[r]
        if r != cur_r:
            proj.set_robot(rb)
            inflated = S.Robot(rb.joints, rb.ee, rb.spheres.copy())
            inflated.spheres[:, 4] += 1e-3
            chk.set_robot(inflated)
            chk.set_constraint(S.no_constraint())
            cur_r = r
        chk.set_obstacles(scenes[sc])
        found, k = [], 0
        while len(found) < 2:
            cand = torch.from_numpy(S.uniform_configs(rb, 64, seed * 1_000_003 + 977 * p + k)
                                    .astype(np.float32)).cuda()
            if cons[c].type != 0:
                proj.set_constraint(cons[c])
                res = proj.project_configs(cand, 60)
                cand = res["q"][res["ok"].bool()].contiguous()
            if len(cand):
                v = chk.validate(cand, cand, 2, with_q=False)
                free = cand[v["status"] == 0]
                found += [free[i] for i in range(min(2 - len(found), len(free)))]
            k += 1
            if k > 400:
                raise RuntimeError(f"no collision-free start/goal for problem {p}")
        start[p, :rb.dof] = found[0]
        goal[p, :rb.dof] = found[1]
    proj.close()
    chk.close()
    return start, goal


def batch_timeline(span, sm_count: int):
    """Problems in flight over one batch run, from each problem's start and end on the GPU's
    global timer (cprrtc_batch_spans)."""
    ran = span[:, 1] > 0
    s0, e0 = span[ran, 0].astype(np.float64), span[ran, 1].astype(np.float64)
    t0, t1 = s0.min(), e0.max()
    T = t1 - t0
    ts = t0 + T * np.linspace(0.0, 1.0, 401)
    inflight = np.array([int(((s0 <= t) & (e0 > t)).sum()) for t in ts])
    full = np.nonzero(inflight >= sm_count)[0]
    last_full = ts[full[-1]] if len(full) else t0
    return {"run_ms": float(T) / 1e6,
            "problem_ms_sum": float((e0 - s0).sum()) / 1e6,
            "mean_in_flight": float((e0 - s0).sum() / T),
            "in_flight_at_pct": {str(q): int(inflight[int(q * 4)]) for q in (0, 10, 25, 50, 75, 90, 99)},
            "last_problem_started_at_ms": float(s0.max() - t0) / 1e6,
            "tail_ms_with_fewer_in_flight_than_sms": float(t1 - last_full) / 1e6,
            "note": "problems in flight at fractions of the run; after the last start the queues "
                    "are empty and the run ends with its slowest problems"}


def run_batch(args, world, rank, local):
    import torch
    from paper_2505_06791_gb300 import build
    from paper_2505_06791_gb300.capi import Context
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    seed = 5 + 1000 * rank
    robots, cons, probs, scenes = S.make_batch_mix(args.problems, seed)
    start, goal = gpu_batch_start_goal(robots, cons, probs, scenes, seed, local)
    stream = torch.cuda.Stream(device=dev)
    ctx = Context(local, stream.cuda_stream)
    ctx.set_robot_table(robots)
    ctx.set_constraint_table(cons)
    ctx.set_scene_batch(scenes)
    prm = ctx.plan_params(seed=seed, use_scene_batch=True, **BATCH_PARAMS)
    max_W = max(p[3] for p in probs)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        tuning = ctx.autotune_batch(probs, start, goal, prm, trial_rounds=20)
        tune_s = time.perf_counter() - t0
        out = ctx.alloc_batch_outputs(len(probs), prm, max_W, start)
        ctx.batch_capture(probs, start, goal, prm, out, tuning=tuning)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        for _ in range(args.warmup):
            ctx.batch_replay()
        stream.synchronize()
        ctx.set_timing(True)
        ctx.reset_timing()
        ctx.work_counters(reset=True)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        clocks = ClockSampler(local)
        barrier(world)
        torch.cuda.synchronize()
        clocks.start()
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            ctx.batch_replay()
            ends[k].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        clk = clocks.stop()
        step_ms = [s_.elapsed_time(e) for s_, e in zip(starts, ends)]
        spans = ctx.batch_spans(len(probs))  # the last timed replay
        kms, launches = ctx.kernel_time("plan_batch")
        counters = ctx.work_counters() / max(args.steps, 1)
        ctx.set_timing(False)
    total_ms = max_over_ranks(sum(step_ms), world)
    L = out["path_len"].cpu().numpy()
    wp = out["waypoints"].cpu().numpy()
    ms = out["plan_ms"].cpu().numpy()
    waypoints_step = int(wp.sum())
    value = sum_over_ranks(waypoints_step, world) * args.steps / (total_ms / 1e3)
    # executed FLOPs: dof differs per problem; weight Alg. 1 updates by the mean dof
    mean_dof = float(np.mean([robots[r].dof for r, _, _, _ in probs]))
    upd, chains, tf, ps, pb, pc = [float(x) for x in counters[:6]]
    flops = (upd * flops_waypoint_iter(round(mean_dof)) + chains * mean_dof * F_CHAIN_JOINT
             + tf * F_SPHERE_FK + ps * F_PAIR_SPHERE + pb * F_PAIR_BOX + pc * F_PAIR_CAPSULE)
    # the autotuned launch shapes against the library's fixed default (as many CTAs as fit,
    # obstacles staged when they fit, one warp per motion): same graph form, inputs and flush
    from paper_2505_06791_gb300.capi import default_tuning
    with torch.cuda.stream(stream):
        out_d = ctx.alloc_batch_outputs(len(probs), prm, max_W, start)
        ctx.batch_capture(probs, start, goal, prm, out_d, tuning=default_tuning())
        ctx.batch_replay()
        ev_d = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
        barrier(world)
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev_d[k][0].record(stream)
            ctx.batch_replay()
            ev_d[k][1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
    d_ms = max_over_ranks(sum(x.elapsed_time(y) for x, y in ev_d), world) / args.steps
    same_d = all(np.array_equal(out_d[k].cpu().numpy(), out[k].cpu().numpy())
                 for k in ("path_len", "rounds", "waypoints"))
    vs_default = {"default_ms_per_step": d_ms, "autotuned_ms_per_step": total_ms / args.steps,
                  "speedup": d_ms / (total_ms / args.steps), "identical_results": same_d}
    del out_d
    # end to end through the C ABI with pinned host buffers
    h_start = start.cpu().pin_memory()
    h_goal = goal.cpu().pin_memory()
    h_out = {k: (torch.empty(v.shape, dtype=v.dtype).pin_memory() if v is not None else None)
             for k, v in out.items()}
    ctx.plan_batch(probs, h_start, h_goal, prm, tuning=tuning, out=h_out)
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        ctx.plan_batch(probs, h_start, h_goal, prm, tuning=tuning, out=h_out)
    e2e_s = time.perf_counter() - t0
    peaks = load_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak, peak_note = fp32_peak(ctx, sm_count, peaks)
    avg_s = kms / 1e3 / max(launches, 1)
    achieved = flops / avg_s / 1e12
    solved = L > 0
    classes = {}
    for (r, c, sc, W) in probs:
        key = f"{['none', 'roll-pitch', 'z-plane'][c]}/W{W}"
        classes[key] = classes.get(key, 0) + 1
    rounds_b = out["rounds"].cpu().numpy()
    # what ends the replay: the problems that run longest (usually to the round cap)
    slow = np.argsort(-ms)[:5]
    critical = {"slowest_problem_ms": float(ms.max()), "step_ms": total_ms / args.steps,
                "slowest": [{"class": f"{['none', 'roll-pitch', 'z-plane'][probs[p][1]]}/W{probs[p][3]}",
                             "dof": int(robots[probs[p][0]].dof),
                             "obstacles": int(len(scenes[probs[p][2]].sph) + len(scenes[probs[p][2]].box)
                                              + len(scenes[probs[p][2]].cap)),
                             "rounds": int(rounds_b[p]), "solved": bool(L[p] > 0),
                             "plan_ms": float(ms[p])} for p in slow],
                "timeline": batch_timeline(spans, torch.cuda.get_device_properties(dev).multi_processor_count),
                "note": "the replay lasts as long as its slowest problem's rounds: the step is "
                        "bound by that critical path, and the SMs idle as the other problems end"}
    learned = None
    if args.learned:
        with torch.cuda.stream(stream):
            pairs = sorted({(r, c) for (r, c, sc_, W_) in probs if cons[c].type in (1, 2)})
            t0 = time.perf_counter()
            for (r, c) in pairs:   # one network per (robot, constraint), trained untimed
                ctx.set_robot(robots[r])
                ctx.set_constraint(cons[c])
                train_warm_network(ctx, robots[r], 40 + 17 * r + 5 * c + 1000 * rank, dev,
                                   args.train_epochs, stream)
                ctx.batch_adopt_network(r, c)
            train_total_s = time.perf_counter() - t0
            ctx.set_plan_warm_start(WS_REFINE)
            out_w = ctx.alloc_batch_outputs(len(probs), prm, max_W, start)
            ctx.batch_capture(probs, start, goal, prm, out_w, tuning=tuning)
            for _ in range(args.warmup):
                ctx.batch_replay()
            ctx.work_counters(reset=True)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            barrier(world)
            torch.cuda.synchronize()
            for k in range(args.steps):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                ctx.batch_replay()
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            barrier(world)
            w_ms = max_over_ranks(sum(x.elapsed_time(y) for x, y in ev), world)
            wcnt = ctx.work_counters() / max(args.steps, 1)
            ctx.set_plan_warm_start(0)
        Lw = out_w["path_len"].cpu().numpy()
        msw = out_w["plan_ms"].cpu().numpy()
        sw = Lw > 0
        learned = {
            "ms_per_step": w_ms / args.steps,
            "value": sum_over_ranks(int(out_w["waypoints"].sum().item()), world) * args.steps / (w_ms / 1e3),
            "p50_plan_ms": float(np.percentile(msw[sw], 50)) if sw.any() else None,
            "p99_plan_ms": float(np.percentile(msw[sw], 99)) if sw.any() else None,
            "success_rate": float(sw.mean()),
            "extend_motions_warm_started_per_step": float(wcnt[6]),
            "warm_segments_accepted_per_step": float(wcnt[7]),
            "networks": [{"robot_dof": int(robots[r].dof),
                          "constraint": ["none", "roll-pitch", "z-plane"][cons[c].type]} for r, c in pairs],
            "training_s": train_total_s,
            "note": "one network per (robot, constraint) pair, trained on 2^20 pairs from "
                    "cprrtc_project_configs; extend motions of those problems warm-started, "
                    "plain Alg. 1 as judge and fallback; unconstrained problems unchanged",
        }
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched uneven serving mix: mixed DOF, obstacle counts, constraints and W in one CUDA-graph launch",
                   "problems": len(probs), "dof": [6, 7, 8],
                   "obstacles_per_problem": "log-uniform [10, 5000], 50/30/20 spheres/boxes/"
                                            "capsules, sizes x min(1, (200/n)^(1/3))",
                   "constraints": ["none", "roll-pitch", "z-plane"], "W": [16, 32, 64],
                   "max_rounds": BATCH_PARAMS["max_rounds"],
                   "workers_per_problem": BATCH_PARAMS["workers"],
                   "recipe_departure": "obstacle sizes shrink by (200/n)^(1/3) above 200 obstacles "
                                       "(the mix names counts, not sizes; full-size primitives at "
                                       "thousands per scene leave few collision-free starts); one "
                                       "CUDA graph of six concurrent class kernels (constraint type "
                                       "x W class) instead of a single persistent kernel",
                   "l2": "flushed (256 MB write) between steps",
                   "parallelism": f"replicas x{world}"},
        "p50_plan_ms": float(np.percentile(ms[solved], 50)) if solved.any() else None,
        "p99_plan_ms": float(np.percentile(ms[solved], 99)) if solved.any() else None,
        "p50_plan_ms_all": float(np.percentile(ms, 50)),
        "p99_plan_ms_all": float(np.percentile(ms, 99)),
        "success_rate": float(solved.mean()),
        "learned_vs_plain": {"plain": {"p50_plan_ms": float(np.percentile(ms[solved], 50)) if solved.any() else None,
                                       "p99_plan_ms": float(np.percentile(ms[solved], 99)) if solved.any() else None,
                                       "success_rate": float(solved.mean()),
                                       "ms_per_step": total_ms / args.steps},
                             "learned": learned},
        "critical_path": critical,
        "waypoints_per_step": waypoints_step,
        "classes": classes,
        "tuning": tuning.as_dict(), "autotune_s": tune_s, "autotuned_vs_default": vs_default,
        "e2e": {"value": waypoints_step * e2e_steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": 2 * len(probs) * 8 * 4,
                "d2h_bytes_per_step": sum(v.numel() * v.element_size()
                                          for v in h_out.values() if v is not None)},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "plan_batch_kernel (6 classes, one graph)",
                     "flop_per_launch": flops, "avg_launch_ms": avg_s * 1e3,
                     "peak_note": peak_note},
        "gpu_launches": int(launches) * sum(1 for v in classes.values() if v),
        "clocks": clk,
    }
    return line, None


def init_dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("CPRRTC_BENCH_GLOO") is None else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x, world, op):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, world):
    """The slowest rank's time (the job's time)."""
    import torch.distributed as dist
    return x if world == 1 else _reduce(x, world, dist.ReduceOp.MAX)


def sum_over_ranks(x, world):
    """Units processed by all ranks (each rank draws its own seeded inputs)."""
    import torch.distributed as dist
    return x if world == 1 else _reduce(x, world, dist.ReduceOp.SUM)


def run_validate(args, world, rank, local):
    import torch
    from paper_2505_06791_gb300 import build
    from paper_2505_06791_gb300.capi import Context
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    rb, sc, c, n, W = validation_workload()
    ctx = Context(local, stream.cuda_stream)
    ctx.set_robot(rb)
    ctx.set_obstacles(sc)
    ctx.set_constraint(c)
    with torch.cuda.stream(stream):
        # each rank validates its own seeded batch (weak scaling, no collective)
        q0 = manifold_starts_gpu(ctx, rb, n, 10_000 + 97 * rank)
        q1 = torch.from_numpy(S.uniform_configs(rb, n, 20_000 + 97 * rank).astype(np.float32)).to(dev)
        out = ctx.alloc_validate_outputs(n, W, q0)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        for _ in range(args.warmup):
            ctx.validate(q0, q1, W, out=out)
        stream.synchronize()
        ctx.set_timing(True)
        ctx.reset_timing()
        ctx.work_counters(reset=True)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        clocks = ClockSampler(local)
        barrier(world)
        torch.cuda.synchronize()
        clocks.start()
        for k in range(args.steps):
            flush.fill_(float(k))            # evict L2 between steps (write > L2 size)
            starts[k].record(stream)
            ctx.validate(q0, q1, W, out=out)
            ends[k].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        clk = clocks.stop()
        step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        kms, launches = ctx.kernel_time("validate")
        counters = ctx.work_counters() / max(args.steps, 1)
        ctx.set_timing(False)
    total_ms = max_over_ranks(sum(step_ms), world)
    st = out["status"].cpu().numpy()
    ff = out["first_fail"].cpu().numpy()
    it = out["iters"].cpu().numpy()
    nominal, cc_wp = algorithmic_flops(rb.dof, W, len(rb.spheres),
                                       (len(sc.sph), len(sc.box), len(sc.cap)), st, ff, it)
    flops = executed_flops(rb.dof, counters)
    waypoints = n * W * args.steps * world
    value = waypoints / (total_ms / 1e3)
    peaks = load_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak, peak_note = fp32_peak(ctx, sm_count, peaks)

    # throughput sweep of the same distribution at sizes that fill the GPU (256 motions are
    # less than one wave of 152 SMs)
    sweep = []
    with torch.cuda.stream(stream):
        for n_s in [int(x) for x in args.sweep.split(",") if x]:
            a0 = manifold_starts_gpu(ctx, rb, n_s, 30_000 + 97 * rank)
            a1 = torch.from_numpy(S.uniform_configs(rb, n_s, 40_000 + 97 * rank).astype(np.float32)).to(dev)
            o_s = ctx.alloc_validate_outputs(n_s, W, a0)
            for _ in range(args.warmup):
                ctx.validate(a0, a1, W, out=o_s)
            stream.synchronize()
            ctx.set_timing(True)
            ctx.reset_timing()
            ctx.work_counters(reset=True)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            barrier(world)
            torch.cuda.synchronize()
            for k in range(args.steps):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                ctx.validate(a0, a1, W, out=o_s)
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            barrier(world)
            ms_s = max_over_ranks(sum(x.elapsed_time(y) for x, y in ev), world)
            k_ms, k_n = ctx.kernel_time("validate")
            cnt = ctx.work_counters() / max(args.steps, 1)
            ctx.set_timing(False)
            st_s = o_s["status"].cpu().numpy()
            ff_s = o_s["first_fail"].cpu().numpy()
            it_s = o_s["iters"].cpu().numpy()
            _, cc_s = algorithmic_flops(rb.dof, W, len(rb.spheres),
                                        (len(sc.sph), len(sc.box), len(sc.cap)), st_s, ff_s, it_s)
            k_s = k_ms / 1e3 / max(k_n, 1)
            ach = executed_flops(rb.dof, cnt) / k_s / 1e12
            sweep.append({"motions": n_s, "value": n_s * W * args.steps * world / (ms_s / 1e3),
                          "ms_per_step": ms_s / args.steps,
                          "evaluated_waypoints_per_s": cc_s * args.steps * world / (ms_s / 1e3),
                          "validate_kernel_ms": k_s * 1e3, "achieved_tflops": ach,
                          "frac": ach / peak, "mean_iters": float(it_s.mean()),
                          "proj_fail": int((st_s == 1).sum()), "collision": int((st_s == 2).sum())})
            del a0, a1, o_s

    # end to end through the C ABI with pinned host buffers
    h_q0 = q0.cpu().pin_memory()
    h_q1 = q1.cpu().pin_memory()
    h_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()}
    for _ in range(2):
        ctx.validate(h_q0, h_q1, W, out=h_out)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.validate(h_q0, h_q1, W, out=h_out)
    e2e_s = time.perf_counter() - t0
    h2d = 2 * n * rb.dof * 4
    d2h = sum(v.numel() * v.element_size() for v in h_out.values())
    e2e = {"value": n * W * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}

    avg_kernel_s = kms / 1e3 / max(launches, 1)
    achieved = flops / avg_kernel_s / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "plain batched constrained motion validation: 7-DOF arm, obstacle spheres in a 1.2 m cube, roll-pitch",
                   "motions": n, "W": W, "dof": rb.dof, "robot_spheres": len(rb.spheres),
                   "obstacles": {"spheres": len(sc.sph)}, "constraint": "roll-pitch",
                   "max_iters": c.max_iters, "l2": "flushed (256 MB write) between steps",
                   "parallelism": f"replicas x{world}"},
        "outcomes": {"valid": int((st == 0).sum()), "proj_fail": int((st == 1).sum()),
                     "collision": int((st == 2).sum()), "mean_iters": float(it.mean()),
                     "cc_waypoints": cc_wp},
        "evaluated_waypoints_per_s": cc_wp * args.steps * world / (total_ms / 1e3),
        "evaluated_note": "waypoints that went through projection, FK and CC: all W of a valid "
                          "motion, up to the first colliding one of a colliding motion, none of "
                          "a motion that failed projection",
        "sweep": sweep,
        "e2e": e2e,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "validate_kernel", "flop_per_launch": flops,
                     "avg_launch_ms": avg_kernel_s * 1e3,
                     "peak_note": peak_note},
        "all_pairs_equivalent": {"flop_per_launch": nominal,
                                 "tflops": nominal / avg_kernel_s / 1e12},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    return line, (rb, sc, c, n, W, q0.cpu().numpy(), q1.cpu().numpy())


# ---- early termination ablation over obstacle density -----------------------------------------

EE_N, EE_W = 4096, 32


def run_earlyexit(args, world, rank, local):
    """The paper's early termination (Sec. IV) against checking every waypoint and candidate,
    on planner-like motions (0.3 rad, roll-pitch) among 24 axis-aligned boxes cut into 1, 10
    and 100 pieces (same occupied volume, 24 to 2400 primitives; the density scaling of
    Sec. V-A). Outputs must be identical with and without early exit."""
    import torch
    from paper_2505_06791_gb300 import build
    from paper_2505_06791_gb300.capi import Context
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    rb, c = S.make_arm7(1), S.roll_pitch(20)
    n, W = EE_N, EE_W
    ctx = Context(local, stream.cuda_stream)
    ctx.set_robot(rb)
    ctx.set_constraint(c)
    rows = []
    total_ms_on = 0.0
    with torch.cuda.stream(stream):
        q0 = manifold_starts_gpu(ctx, rb, n, 30_000 + 97 * rank)
        q1 = torch.from_numpy(S.nearby_configs(rb, q0.cpu().numpy(), 0.3,
                                               31_000 + 97 * rank).astype(np.float32)).to(dev)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        clocks = ClockSampler(local)
        clocks.start()
        for split in (1, 10, 100):
            sc = S.make_subdivided_boxes(40 + rank, 24, split)
            ctx.set_obstacles(sc)
            res = {}
            for early in (True, False):
                ctx.set_early_exit(early)
                out = ctx.alloc_validate_outputs(n, W, q0)
                for _ in range(args.warmup):
                    ctx.validate(q0, q1, W, out=out)
                stream.synchronize()
                ctx.work_counters(reset=True)
                starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
                ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
                barrier(world)
                torch.cuda.synchronize()
                for k in range(args.steps):
                    flush.fill_(float(k))
                    starts[k].record(stream)
                    ctx.validate(q0, q1, W, out=out)
                    ends[k].record(stream)
                torch.cuda.synchronize()
                barrier(world)
                ms = max_over_ranks(sum(s_.elapsed_time(e) for s_, e in zip(starts, ends)), world)
                cnt = ctx.work_counters() / max(args.steps, 1)
                res[early] = dict(ms=ms / args.steps, tests=float(cnt[3:].sum()),
                                  out={k: v.cpu().numpy() for k, v in out.items()})
            ctx.set_early_exit(True)
            same = all(np.array_equal(res[True]["out"][k], res[False]["out"][k])
                       for k in ("status", "first_fail", "q"))
            st = res[True]["out"]["status"]
            if split == 100:
                total_ms_on = res[True]["ms"] * args.steps
            rows.append({"boxes": len(sc.box), "early_exit_ms": res[True]["ms"],
                         "no_early_exit_ms": res[False]["ms"],
                         "speedup": res[False]["ms"] / res[True]["ms"],
                         "tests_early_exit": res[True]["tests"],
                         "tests_no_early_exit": res[False]["tests"],
                         "identical_outputs": bool(same),
                         "collision_rate": float((st == 2).mean())})
        clk = clocks.stop()
    value = sum_over_ranks(n * W * args.steps, world) / (max_over_ranks(total_ms_on, world) / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_on / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "early-termination ablation: 24 boxes cut into 1/10/100",
                   "motions": n, "W": W, "dof": rb.dof, "constraint": "roll-pitch",
                   "motion": "0.3 rad from on-manifold starts",
                   "value_from": "early exit on, 2400 boxes",
                   "l2": "flushed (256 MB write) between steps",
                   "parallelism": f"replicas x{world}"},
        "densities": rows,
        "gpu_launches": int(args.steps * 6),
        "clocks": clk,
    }
    return line, None


# ---- the paper's naive baseline: sequential projection inside the same planner -------------

NAIVE_N = 304


def run_naive(args, world, rank, local):
    """cpRRTC-Naive against cpRRTC-Parallel (Sec. V): the full planner (7-DOF arm, 200 mixed obstacles per problem) on 304
    problems (one wave of 2 per SM), once with Alg. 1 and once with the sequential
    projection; success, plan time and validated waypoints per second for each."""
    import torch
    from paper_2505_06791_gb300 import build
    from paper_2505_06791_gb300.capi import Context
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rb, c = S.make_arm7(1), S.roll_pitch(20)
    n = NAIVE_N
    seed = 7 + 1000 * rank
    scenes = planner_scenes(n, seed)
    start, goal = gpu_start_goal(rb, c, scenes, seed, local)
    stream = torch.cuda.Stream(device=dev)
    ctx = Context(local, stream.cuda_stream)
    ctx.set_robot(rb)
    ctx.set_constraint(c)
    ctx.set_scene_batch(scenes)
    prm = ctx.plan_params(seed=seed, **PLAN_PARAMS)
    modes = {}
    with torch.cuda.stream(stream):
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        clocks = ClockSampler(local)
        clocks.start()
        for name, seq in (("parallel", False), ("naive", True)):
            ctx.set_projection(seq)
            out = ctx.alloc_plan_outputs(n, prm, start, edges=False)
            for _ in range(args.warmup):
                ctx.plan(start, goal, prm, out=out)
            stream.synchronize()
            starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            barrier(world)
            torch.cuda.synchronize()
            for k in range(args.steps):
                flush.fill_(float(k))
                starts[k].record(stream)
                ctx.plan(start, goal, prm, out=out)
                ends[k].record(stream)
            torch.cuda.synchronize()
            barrier(world)
            ms = max_over_ranks(sum(s_.elapsed_time(e) for s_, e in zip(starts, ends)), world)
            L = out["path_len"].cpu().numpy()
            pm = out["plan_ms"].cpu().numpy()
            wp = int(out["waypoints"].cpu().numpy().sum())
            work = out["work"].cpu().numpy()
            solved = L > 0
            modes[name] = {
                "ms_per_step": ms / args.steps,
                "value": sum_over_ranks(wp, world) * args.steps / (ms / 1e3),
                "success_rate": float(solved.mean()),
                "p50_plan_ms": float(np.median(pm[solved])) if solved.any() else None,
                "mean_plan_ms_solved": float(pm[solved].mean()) if solved.any() else None,
                "mean_rounds": float(out["rounds"].cpu().numpy().mean()),
                "projection_updates_per_waypoint": float(work[:, 0].sum() / max(wp, 1)),
            }
        ctx.set_projection(False)
        clk = clocks.stop()
    par, nv = modes["parallel"], modes["naive"]
    line = {
        "metric": METRIC, "value": par["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": par["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "cpRRTC-Parallel vs cpRRTC-Naive projection inside the full planner (7-DOF arm, 200 mixed obstacles, roll-pitch)",
                   "problems": n, "W": PLAN_PARAMS["W"], "range": PLAN_PARAMS["range_"],
                   "max_rounds": PLAN_PARAMS["max_rounds"], "constraint": "roll-pitch",
                   "l2": "flushed (256 MB write) between steps",
                   "parallelism": f"replicas x{world}"},
        "modes": modes,
        "parallel_vs_naive": {
            "success_rate_delta": par["success_rate"] - nv["success_rate"],
            "mean_solved_plan_ms_ratio": (nv["mean_plan_ms_solved"] / par["mean_plan_ms_solved"])
            if par["mean_plan_ms_solved"] and nv["mean_plan_ms_solved"] else None,
            "paper": "Parallel 1.1x faster, success +19 % (Sec. V, RTX 5090, MotionBenchMaker)"},
        "gpu_launches": int(2 * args.steps),
        "clocks": clk,
    }
    return line, None


# ---- obstacle-rich scene: collision checking in GEMM form ---------------------------------------------

CC_N, CC_W = 4096, 64


def point_cloud_workload(seed=3):
    """8-DOF arm (7-DOF arm on a 0..0.4 m prismatic torso, 120 spheres), 4096 obstacle
    spheres of radius 0.02 m on the surfaces of 12 random boxes, end effector on z = 0.9 m."""
    return S.make_arm8(1), S.make_box_surface_cloud(seed), S.z_plane(0.9)


def near_ends(q0, rb, half_width, seed):
    """Planner-like motion ends: each start moved by U[-w, w] per joint, clipped to the limits."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    d = (torch.rand(q0.shape, generator=g) * 2 - 1) * half_width
    lo = torch.tensor(rb.lo, dtype=torch.float32)
    hi = torch.tensor(rb.hi, dtype=torch.float32)
    return torch.maximum(torch.minimum(q0.cpu() + d, hi), lo).to(q0.device).contiguous()


def run_gemmcc(args, world, rank, local):
    """Validation of 4096 motions x 64 waypoints with the exact collision check and with the
    GEMM form (TF32 and BF16 contraction + exact recheck); outputs compared across modes.
    Two motion sets on the same scene: ends uniform in the joint limits (the configuration;
    most motions fail the projection before any collision check), and planner-like ends
    within 0.3 rad of the start (most motions reach the collision check)."""
    import torch
    from paper_2505_06791_gb300 import build
    from paper_2505_06791_gb300.capi import Context
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    rb, sc, c = point_cloud_workload()
    n, W = (CC_N if args.problems == PLAN_N else args.problems), CC_W
    ctx = Context(local, stream.cuda_stream)
    ctx.set_robot(rb)
    ctx.set_obstacles(sc)
    ctx.set_constraint(c)
    peaks = load_peaks()
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    n_obs, n_rs = len(sc.sph), len(rb.spheres)
    n_tiles = (n_obs + 255) // 256

    def measure(q0, q1, flush):
        modes = {}
        for name, mode in (("exact", 0), ("gemm_tf32", 1), ("gemm_bf16", 2)):
            ctx.set_cc_mode(mode, 0.005)
            out = ctx.alloc_validate_outputs(n, W, q0)
            for _ in range(args.warmup):
                ctx.validate(q0, q1, W, out=out)
            stream.synchronize()
            ctx.cc_stats(reset=True)
            ctx.set_timing(True)
            ctx.reset_timing()
            starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            barrier(world)
            torch.cuda.synchronize()
            for k in range(args.steps):
                flush.fill_(float(k))            # evict L2 between steps (write > L2 size)
                starts[k].record(stream)
                ctx.validate(q0, q1, W, out=out)
                ends[k].record(stream)
            torch.cuda.synchronize()
            barrier(world)
            ms = max_over_ranks(sum(s_.elapsed_time(e) for s_, e in zip(starts, ends)), world)
            kv = ctx.kernel_time("validate")
            kg = ctx.kernel_time("gemm_cc")
            ctx.set_timing(False)
            bound, rechecks = ctx.cc_stats(reset=True)
            modes[name] = dict(ms=ms, kv=kv, kg=kg, bound=bound, rechecks=rechecks / max(args.steps, 1),
                               out={k: v.cpu().numpy() for k, v in out.items()})
        ctx.set_cc_mode(0)
        ex = modes["exact"]["out"]
        st, ff = ex["status"], ex["first_fail"]
        # waypoint tiles the GEMM form evaluates: every waypoint of a collision-free projected
        # motion, and up to the first colliding waypoint + 1 of a colliding one
        tiles = int(np.where(st == 0, W, np.where(st == 2, np.minimum(ff + 2, W), 0)).sum())
        # algorithmic work: 16 FLOP per (robot sphere, obstacle) pair of an evaluated
        # waypoint (the distance as an 8-term augmented dot product, 2 x 8); the MMAs as
        # issued (128 padded rows, 256-column tiles, K = 16 hi/lo-split terms) are counted
        # separately
        tensor_flop = tiles * n_rs * n_obs * 16
        issued_flop = tiles * 128 * n_tiles * 256 * 2 * 16
        wps = n * W * args.steps * world
        summary = {}
        for name, m in modes.items():
            o = m["out"]
            same = bool(np.array_equal(o["status"], st) and np.array_equal(o["first_fail"], ff)
                        and np.array_equal(o["q"], ex["q"]))
            entry = {"value": wps / (m["ms"] / 1e3), "ms_per_step": m["ms"] / args.steps,
                     "evaluated_waypoints_per_s": tiles * args.steps * world / (m["ms"] / 1e3),
                     "validate_kernel_ms": m["kv"][0] / max(m["kv"][1], 1), "identical_to_exact": same}
            if name != "exact":
                g_ms = m["kg"][0] / max(m["kg"][1], 1)
                peak = bf16_peak if name == "gemm_bf16" else bf16_peak / 2.0
                entry.update({"gemm_cc_kernel_ms": g_ms, "error_bound_m2": m["bound"],
                              "exact_rechecks_per_step": m["rechecks"],
                              "tensor_tflops": tensor_flop / (g_ms / 1e3) / 1e12,
                              "issued_mma_tflops": issued_flop / (g_ms / 1e3) / 1e12,
                              "tensor_peak_tflops": peak,
                              "peak_note": "BF16 measured (MEASURED_PEAKS.json bf16_tflops); TF32 = "
                                           "BF16 x 0.5 (nominal dense ratio)" if name == "gemm_tf32"
                                           else "BF16 measured (MEASURED_PEAKS.json bf16_tflops)"})
            summary[name] = entry
        outcomes = {"valid": int((st == 0).sum()), "proj_fail": int((st == 1).sum()),
                    "collision": int((st == 2).sum()), "gemm_waypoint_tiles": tiles}
        return summary, outcomes, tensor_flop, issued_flop, tiles

    with torch.cuda.stream(stream):
        q0 = manifold_starts_gpu(ctx, rb, n, 70_000 + 97 * rank)
        q1 = torch.from_numpy(S.uniform_configs(rb, n, 80_000 + 97 * rank).astype(np.float32)).to(dev)
        q1n = near_ends(q0, rb, 0.3, 81_000 + 97 * rank)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        clocks = ClockSampler(local)
        clocks.start()
        summary, outcomes, tensor_flop, issued_flop, tiles = measure(q0, q1, flush)
        near_summary, near_outcomes, near_flop, near_issued, near_tiles = measure(q0, q1n, flush)
        clk = clocks.stop()
    best = max(("gemm_tf32", "gemm_bf16"), key=lambda k: summary[k]["value"])
    gcc_tile_bytes = profiled_traffic_per_unit("gemm_cc_kernel_point_cloud_4096.md", "traffic_per_waypoint_tile_bytes")
    b = summary[best]
    nb = near_summary["gemm_bf16"]
    line = {
        "metric": METRIC, "value": b["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": b["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": f"{best[5:]} contraction, f32 recheck",
        "data": "synthetic",
        "config": {"workload": "obstacle-rich scene, collision check in GEMM form: 8-DOF arm, point-cloud sphere obstacles, z-plane",
                   "motions": n, "W": W, "dof": rb.dof, "robot_spheres": n_rs,
                   "obstacles": {"spheres": n_obs, "radius": 0.02},
                   "constraint": "z-plane 0.9 m", "guard_m": 0.005, "motion_ends": "uniform in the joint limits",
                   "l2": "flushed (256 MB write) between steps", "parallelism": f"replicas x{world}"},
        "modes": summary,
        "outcomes": outcomes,
        "planner_like": {"motion_ends": "start + U[-0.3, 0.3] rad per joint, clipped",
                         "modes": near_summary, "outcomes": near_outcomes,
                         "roofline_bf16": {"bound": "tensor", "achieved": nb["tensor_tflops"],
                                           "peak": nb["tensor_peak_tflops"], "unit": "TFLOP/s",
                                           "frac": nb["tensor_tflops"] / nb["tensor_peak_tflops"],
                                           "flop_per_launch": near_flop,
                                           "issued_mma_flop_per_launch": near_issued,
                                           "avg_launch_ms": nb["gemm_cc_kernel_ms"]}},
        "roofline": {"bound": "tensor", "achieved": b["tensor_tflops"], "peak": b["tensor_peak_tflops"],
                     "unit": "TFLOP/s", "frac": b["tensor_tflops"] / b["tensor_peak_tflops"],
                     "traffic": (None if gcc_tile_bytes is None or best != "gemm_bf16"
                                 else gcc_tile_bytes * tiles),
                     "traffic_note": "ncu DRAM bytes per waypoint tile of a 512-motion BF16 capture "
                                     "(profiles/gemm_cc_kernel_point_cloud_4096.md) x waypoint tiles",
                     "kernel": "gemm_cc_kernel",
                     "flop_per_launch": tensor_flop,
                     "flop_note": "16 FLOP per (robot sphere, obstacle) pair of each evaluated waypoint",
                     "issued_mma_flop_per_launch": issued_flop,
                     "avg_launch_ms": b["gemm_cc_kernel_ms"]},
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
    }
    return line, (rb, sc, c, 64, W, q0[:64].cpu().numpy(), q1[:64].cpu().numpy())


# ---- learned warm start -------------------------------------------------------

WS_MOTIONS = 16384
WS_W = 32
WS_TRAIN = 1 << 20
WS_EPOCHS = 10
WS_REFINE = 5


def train_warm_network(ctx, rb, seed, dev, epochs, stream):
    """The warm-start network of the context's robot and constraint, trained (untimed) on 2^20
    (uniform configuration -> its projection) pairs from cprrtc_project_configs; held-out
    loss before and after on 16384 more pairs."""
    import torch
    t0 = time.perf_counter()
    qs, ts, k = [], [], 0
    while sum(len(x) for x in qs) < WS_TRAIN + 16384:
        q = torch.from_numpy(S.uniform_configs(rb, 1 << 19, seed * 7919 + k).astype(np.float32)).to(dev)
        r = ctx.project_configs(q, 60)
        ok = r["ok"].bool()
        qs.append(q[ok])
        ts.append(r["q"][ok])
        k += 1
    q_all, t_all = torch.cat(qs), torch.cat(ts)
    q_tr, t_tr = q_all[:WS_TRAIN].contiguous(), t_all[:WS_TRAIN].contiguous()
    q_ho = q_all[WS_TRAIN:WS_TRAIN + 16384].contiguous()
    t_ho = t_all[WS_TRAIN:WS_TRAIN + 16384].contiguous()
    stream.synchronize()
    pairs_s = time.perf_counter() - t0
    ctx.mlp_init(seed)
    held0, _ = ctx.mlp_grad(q_ho, t_ho)
    t0 = time.perf_counter()
    losses = ctx.mlp_train(q_tr, t_tr, batch=1024, epochs=epochs, lr=1e-3, seed=seed)
    train_s = time.perf_counter() - t0
    held1, _ = ctx.mlp_grad(q_ho, t_ho)
    zero_loss = float(0.5 * ((t_ho - q_ho) ** 2).sum(1).mean())
    return dict(pairs_s=pairs_s, train_s=train_s, losses=losses, held0=held0, held1=held1,
                zero_loss=zero_loss)


def mlp_flops_per_row(dof: int, hidden: int = 256) -> int:
    """Multiply-adds of the warm-start network per row, x 2."""
    return 2 * (dof * hidden + 2 * hidden * hidden + hidden * dof)


def warm_start_workload(seed=4):
    """7-DOF arm (59 spheres), roll/pitch constraint, one config-2 scene (100 spheres, 60
    boxes, 40 capsules)."""
    rb = S.make_arm7(1)
    c = S.roll_pitch(20)
    sc = S.make_planning_scene(4_000_000 + seed)
    return rb, sc, c


def run_warmstart(args, world, rank, local):
    """Plain Alg. 1 validation against the learned warm start on the same motions: the
    network is trained first (untimed) on 2^20 (uniform configuration -> its projection)
    pairs, the projection done by the library's cprrtc_project_configs."""
    import torch
    from paper_2505_06791_gb300 import build
    from paper_2505_06791_gb300.capi import Context
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    rb, sc, c = warm_start_workload()
    n, W = (WS_MOTIONS if args.problems == PLAN_N else args.problems), WS_W
    ctx = Context(local, stream.cuda_stream)
    ctx.set_robot(rb)
    ctx.set_obstacles(sc)
    ctx.set_constraint(c)
    seed = 40 + 1000 * rank
    with torch.cuda.stream(stream):
        tr = train_warm_network(ctx, rb, seed, dev, args.train_epochs, stream)
        pairs_s, train_s, losses = tr["pairs_s"], tr["train_s"], tr["losses"]
        held0, held1, zero_loss = tr["held0"], tr["held1"], tr["zero_loss"]

        q0 = manifold_starts_gpu(ctx, rb, n, 50_000 + 97 * rank)
        q1 = torch.from_numpy(S.uniform_configs(rb, n, 60_000 + 97 * rank).astype(np.float32)).to(dev)
        out_p = ctx.alloc_validate_outputs(n, W, q0)
        out_w = ctx.alloc_validate_outputs(n, W, q0)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        for _ in range(args.warmup):
            ctx.validate(q0, q1, W, out=out_p)
            ctx.validate_ws(q0, q1, W, WS_REFINE, out=out_w)
        stream.synchronize()

        def timed(fn):
            ctx.set_timing(True)
            ctx.reset_timing()
            starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            barrier(world)
            torch.cuda.synchronize()
            for k_ in range(args.steps):
                flush.fill_(float(k_))        # evict L2 between steps (write > L2 size)
                starts[k_].record(stream)
                fn()
                ends[k_].record(stream)
            torch.cuda.synchronize()
            barrier(world)
            ms = max_over_ranks(sum(s_.elapsed_time(e) for s_, e in zip(starts, ends)), world)
            kt = {name: ctx.kernel_time(name) for name in ("validate", "mlp_infer")}
            ctx.set_timing(False)
            return ms, kt

        clocks = ClockSampler(local)
        clocks.start()
        ms_plain, kt_plain = timed(lambda: ctx.validate(q0, q1, W, out=out_p))
        ms_ws, kt_ws = timed(lambda: ctx.validate_ws(q0, q1, W, WS_REFINE, out=out_w))
        # the planner's motions (steering range 0.3 rad, as in the full planner and the uneven batch):
        # plain against warm start on the same starts
        q1s = torch.from_numpy(S.nearby_configs(rb, q0.cpu().numpy(), 0.3,
                                                61_000 + 97 * rank).astype(np.float32)).to(dev)
        out_ps = ctx.alloc_validate_outputs(n, W, q0)
        out_ws = ctx.alloc_validate_outputs(n, W, q0)
        for _ in range(args.warmup):
            ctx.validate(q0, q1s, W, out=out_ps)
            ctx.validate_ws(q0, q1s, W, WS_REFINE, out=out_ws)
        ms_ps, _ = timed(lambda: ctx.validate(q0, q1s, W, out=out_ps))
        ms_wss, _ = timed(lambda: ctx.validate_ws(q0, q1s, W, WS_REFINE, out=out_ws))
        clk = clocks.stop()
    Ps = {k: v.cpu().numpy() for k, v in out_ps.items()}
    Ws_ = {k: v.cpu().numpy() for k, v in out_ws.items()}
    short = {"motion": "0.3 rad from the same starts (planner steering range)",
             "plain_ms_per_step": ms_ps / args.steps, "warm_start_ms_per_step": ms_wss / args.steps,
             "plain_projected": int((Ps["status"] != 1).sum()),
             "warm_start_projected": int((Ws_["status"] != 1).sum()),
             "plain_mean_iters": float(Ps["iters"].astype(float).mean()),
             "warm_start_mean_iters": float(Ws_["iters"].astype(float).mean()),
             "warm_used": float(Ws_["warm"].astype(bool).mean())}

    P = {k: v.cpu().numpy() for k, v in out_p.items()}
    Wr = {k: v.cpu().numpy() for k, v in out_w.items()}
    used = Wr["warm"].astype(bool)
    extra = Wr["iters"].astype(int) - P["iters"].astype(int)
    tried = used | ((~used) & (extra == WS_REFINE))
    p_ok, w_ok = P["status"] != 1, Wr["status"] != 1
    wps = n * W * args.steps * world
    value_ws, value_plain = wps / (ms_ws / 1e3), wps / (ms_plain / 1e3)

    # end to end through the C ABI with pinned host buffers
    h_q0, h_q1 = q0.cpu().pin_memory(), q1.cpu().pin_memory()
    h_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out_w.items()}
    ctx.validate_ws(h_q0, h_q1, W, WS_REFINE, out=h_out)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.validate_ws(h_q0, h_q1, W, WS_REFINE, out=h_out)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": n * W * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 2 * n * rb.dof * 4,
           "d2h_bytes_per_step": sum(v.numel() * v.element_size() for v in h_out.values())}

    peaks = load_peaks()
    infer_ms, infer_launches = kt_ws["mlp_infer"]
    infer_avg_s = infer_ms / 1e3 / max(infer_launches, 1)
    flops_infer = mlp_flops_per_row(rb.dof) * n * W
    mlp_row_bytes = profiled_traffic_per_unit("mlp_fused_kernel_warm_start_16384x32.md", "traffic_per_row_bytes")
    tensor_peak = float(peaks.get("bf16_tflops", 1900.0))
    achieved = flops_infer / infer_avg_s / 1e12
    vk_ms, vk_launches = kt_ws["validate"]
    line = {
        "metric": METRIC, "value": value_ws, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_ws / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16 network, f32 projection",
        "data": "synthetic",
        "config": {"workload": "learned warm start vs plain projection: 7-DOF arm among 200 mixed obstacles, roll-pitch",
                   "motions": n, "W": W, "dof": rb.dof, "robot_spheres": len(rb.spheres),
                   "obstacles": {"spheres": len(sc.sph), "boxes": len(sc.box),
                                 "capsules": len(sc.cap)},
                   "constraint": "roll-pitch", "refine_iters": WS_REFINE,
                   "max_iters": c.max_iters, "l2": "flushed (256 MB write) between steps",
                   "recipe_departure": "the 2^20 training pairs are projections by the library's "
                                       "cprrtc_project_configs, not the oracle's (the bench runs "
                                       "the oracle only in its CPU-baseline leg; the tests train "
                                       "on oracle pairs)",
                   "parallelism": f"replicas x{world}"},
        "plain": {"value": value_plain, "ms_per_step": ms_plain / args.steps,
                  "projected": int(p_ok.sum()), "success_rate": float(p_ok.mean()),
                  "valid": int((P["status"] == 0).sum()),
                  "mean_iters": float(P["iters"].astype(float).mean())},
        "warm_start": {"value": value_ws, "ms_per_step": ms_ws / args.steps,
                       "projected": int(w_ok.sum()), "success_rate": float(w_ok.mean()),
                       "valid": int((Wr["status"] == 0).sum()),
                       "mean_iters": float(Wr["iters"].astype(float).mean()),
                       "mean_iters_on_plain_projected": float(Wr["iters"][p_ok].astype(float).mean())
                       if p_ok.any() else None,
                       "plain_mean_iters_on_plain_projected": float(P["iters"][p_ok].astype(float).mean())
                       if p_ok.any() else None,
                       "warm_used": float(used.mean()), "tried": float(tried.mean()),
                       "fallback_rate": float((tried & ~used).sum() / max(tried.sum(), 1)),
                       "lost": int((p_ok & ~w_ok).sum()),
                       "infer_ms_per_step": infer_avg_s * 1e3,
                       "validate_ms_per_step": vk_ms / max(vk_launches, 1)},
        "planner_like_motions": short,
        "training": {"pairs": WS_TRAIN, "pair_generation_s": pairs_s,
                     "epochs": args.train_epochs, "batch": 1024, "lr": 1e-3, "train_s": train_s,
                     "samples_per_s": args.train_epochs * WS_TRAIN / train_s,
                     "loss_first_last_epoch": [float(losses[0]), float(losses[-1])],
                     "heldout_loss_init_trained": [held0, held1],
                     "heldout_zero_prediction_loss": zero_loss,
                     "pairs_source": "uniform configurations projected by cprrtc_project_configs"},
        "e2e": e2e,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": tensor_peak, "unit": "TFLOP/s",
                     "frac": achieved / tensor_peak,
                     "traffic": (None if mlp_row_bytes is None else mlp_row_bytes * n * W),
                     "traffic_note": "ncu DRAM bytes per row of a 131072-row capture "
                                     "(profiles/mlp_fused_kernel_warm_start_16384x32.md) x rows",
                     "kernel": "mlp_fused_kernel",
                     "flop_per_launch": flops_infer, "avg_launch_ms": infer_avg_s * 1e3,
                     "peak_note": "measured dense BF16 (MEASURED_PEAKS.json bf16_tflops, burst)"},
        "gpu_launches": int(kt_ws["validate"][1] + kt_ws["mlp_infer"][1]),
        "clocks": clk,
    }
    return line, (rb, sc, c, min(n, 2048), W, q0[:2048].cpu().numpy(), q1[:2048].cpu().numpy())


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}


def cpu_baseline_validate(inputs, budget_s=10.0):
    """The FP64 oracle, as it stands, on the host cores over the same motions."""
    import oracle
    rb, sc, c, n, W, q0, q1 = inputs
    orc = oracle.Oracle(rb, sc, c)
    cores = os.cpu_count() or 1
    reps, t0 = 0, time.perf_counter()
    while True:
        orc.validate(q0, q1, W, n_threads=cores)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= 200:
            break
    return {"value": n * W * reps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} passes over the same {n} motions x {W} waypoints "
                      f"({el:.1f} s, {cores} threads)"}


def reference_arm_plan(args, world, rank):
    """The oracle arm on the planner workload: the FP64 oracle's RRT-Connect on the same
    seeded problems (start/goal chosen by the oracle), a bounded sample per step."""
    if rank != 0:
        return None
    import oracle
    rb, c = S.make_arm7(1), S.roll_pitch(20)
    seed = 2
    cores = os.cpu_count() or 1
    n = cores
    scenes = planner_scenes(n, seed)
    starts, goals = [], []
    for p, sc in enumerate(scenes):
        orc = oracle.Oracle(rb, sc, c)
        found = []
        k = 0
        while len(found) < 2:
            for q in S.uniform_configs(rb, 64, seed * 1_000_003 + 977 * p + k):
                ok, qp, _, _ = orc.project_config(q, max_iters=60)
                if ok and orc.config_clearance(qp) > 1e-3:
                    found.append(qp)
                if len(found) == 2:
                    break
            k += 1
        starts.append(found[0])
        goals.append(found[1])
    start, goal = S.f32(np.array(starts)), S.f32(np.array(goals))
    budget = max(2.0, args.cpu_budget / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_plan_sample(rb, c, scenes, start, goal, seed, budget, cores)
    tot_wp, tot_s, ms_all = 0.0, 0.0, []
    for _ in range(args.steps):
        v, ms, n_done, solved, el = oracle_plan_sample(rb, c, scenes, start, goal, seed, budget, cores)
        tot_wp += v * el
        tot_s += el
        ms_all += ms
    value = tot_wp / tot_s
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "full planner, plain form: RRT-Connect on a 7-DOF arm among 200 mixed obstacles per problem, roll-pitch",
                       "problems": n, "dof": rb.dof, "parallelism": "host threads"},
            "p50_plan_ms": float(np.percentile(ms_all, 50)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{cores} problems per step, one per thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def reference_arm(args, world, rank):
    """The oracle arm: the FP64 CPU oracle as it stands, on the same workload and metric."""
    if rank != 0:
        return None
    import oracle
    rb, sc, c, n, W = validation_workload()
    orc = oracle.Oracle(rb, sc, c)
    starts = []
    for q in S.uniform_configs(rb, 4 * n, 10_000):
        ok, qp, _, _ = orc.project_config(q, max_iters=60)
        if ok:
            starts.append(qp)
        if len(starts) == n:
            break
    q0 = S.f32(np.array(starts))
    q1 = S.uniform_configs(rb, n, 20_000)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        orc.validate(q0, q1, W, n_threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.validate(q0, q1, W, n_threads=cores)
    el = time.perf_counter() - t0
    value = n * W * args.steps / el
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "plain batched constrained motion validation: 7-DOF arm, obstacle spheres in a 1.2 m cube, roll-pitch",
                       "motions": n, "W": W, "dof": rb.dof, "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} passes over {n} motions x {W} waypoints"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def run_legs(args):
    """The other configurations, each in a child process with the same steps and warm-up,
    its own JSON line kept whole (a failing leg records its error instead)."""
    legs = {}
    for leg in [x for x in args.legs.split(",") if x]:
        cmd = [sys.executable, os.path.abspath(__file__), "--workload", leg, "--steps", str(args.steps),
               "--warmup", str(args.warmup), "--cpu-budget", "3", "--legs", "none"]
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
            lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
            legs[leg] = json.loads(lines[-1]) if r.returncode == 0 and lines else \
                {"error": f"exit {r.returncode}: {r.stderr.strip()[-300:]}"}
        except (subprocess.TimeoutExpired, ValueError) as e:
            legs[leg] = {"error": str(e)[:300]}
    return legs


def main():
    global PLAN_SLICING
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="plan",
                    choices=["plan", "validate", "batch", "warmstart", "gemmcc", "earlyexit",
                             "naive"])
    ap.add_argument("--problems", type=int, default=PLAN_N)
    ap.add_argument("--max-rounds", type=int, default=None,
                    help="override the planner's round cap (small profiling runs)")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--sweep", default=",".join(str(x) for x in VAL_SWEEP),
                    help="validation workload: motion counts of the throughput sweep")
    ap.add_argument("--learned", type=int, default=1,
                    help="planner workload: also time the learned form (trains the network first)")
    ap.add_argument("--slicing", default=None,
                    help="planner's time-sliced schedule 'first,slice' in rounds (0,0: one CTA "
                         "per problem); default %d,%d" % PLAN_SLICING)
    ap.add_argument("--schedule-ab", type=int, default=1,
                    help="planner workload: also time one CTA per problem without time slicing")
    ap.add_argument("--train-epochs", type=int, default=WS_EPOCHS,
                    help="warm-start training epochs (fewer for profiling runs)")
    ap.add_argument("--legs", default="validate,gemmcc,warmstart,batch,earlyexit,naive",
                    help="with the default planner workload on one GPU: the other configurations, "
                         "each run as its own process and reported under 'legs' ('none' to skip)")
    args = ap.parse_args()
    if args.slicing is not None:
        PLAN_SLICING = tuple(int(x) for x in args.slicing.split(","))
    if args.max_rounds is not None:
        PLAN_PARAMS["max_rounds"] = args.max_rounds
        BATCH_PARAMS["max_rounds"] = args.max_rounds
    world, rank, local = init_dist()
    if args.impl == "reference":
        fn = reference_arm_plan if args.workload == "plan" else reference_arm
        line = fn(args, world, rank)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if args.workload == "plan":
        line, inputs = run_plan(args, world, rank, local)
        baseline = cpu_baseline_plan
    elif args.workload == "batch":
        if args.problems == PLAN_N:
            args.problems = BATCH_N
        line, inputs = run_batch(args, world, rank, local)
        baseline = None
    elif args.workload == "gemmcc":
        line, inputs = run_gemmcc(args, world, rank, local)
        baseline = cpu_baseline_validate
    elif args.workload == "warmstart":
        line, inputs = run_warmstart(args, world, rank, local)
        baseline = cpu_baseline_validate
    elif args.workload == "earlyexit":
        line, inputs = run_earlyexit(args, world, rank, local)
        baseline = None
    elif args.workload == "naive":
        line, inputs = run_naive(args, world, rank, local)
        baseline = None
    else:
        line, inputs = run_validate(args, world, rank, local)
        baseline = cpu_baseline_validate
    if rank == 0:
        if world == 1 and baseline is not None:
            line["cpu_baseline"] = baseline(inputs, args.cpu_budget)
        if args.workload == "plan" and world == 1 and args.legs != "none":
            line["legs"] = run_legs(args)
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
