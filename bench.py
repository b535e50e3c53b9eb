"""Benchmark of the batched HeSP simulator (sim task-events/s, bit-exact).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hesp|reference]

One step = the hot path over one batch: 4,096 candidate partition vectors of
the 32 x 32-tile Cholesky (N = 65536, b = 2048, 5,984 base tasks, split
levels uniform in {0, 1, 2, 3}: DAGs of ~810,000 tasks) drawn on the device
from SplitMix64, then expanded, dependence-analysed and simulated on 32 CPU
+ 2 GPU-type processors (FCFS + EFT-P, write-back caching of the two GPU
memories) in one launch that holds every candidate resident, and reduced on
the device to the batch's best candidate (least makespan, lowest index).
The metric counts one task-event per task scheduled and completed in one
candidate's simulation.

Extra keys of the same run (one GPU): the 8 x 8-tile random-search step on
its two platforms ("random_8x8_two_platforms": 65,536 candidates, 12 CPU +
1 GPU-type and 4 big + 4 LITTLE), and the best makespan reached in 60 s of
GPU time on the 32 x 32-tile problem by plain batched random search, by
surrogate-guided search and by the paper's iterative solver ("search").

N > 1 (torchrun): weak scaling -- rank r simulates its own 4,096 candidates
per step (global indices (step * N + r) * 4096 ...); after the timed loop
the ranks exchange their per-step best (makespan, index) pairs in one
all-gather (16 bytes per rank and step), and rank 0 reports the best over
all ranks; the timed region ends with a barrier and a max over ranks.

--impl reference times the CPU oracle (the plain C implementation the GPU
results are checked against) on the host cores, on a bounded sample of the
same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1602_05510_b300 import workloads as W  # noqa: E402

# the 32 x 32-tile random-search launch
N_TILES, B, N_LEVELS, N_CAND, SEED = 32, 2048, 4, 4096, 4
MAX_LEVEL = N_LEVELS - 1
PLAT = "cfg4"  # 32 CPU + 2 GPU-type processors
TASK_CAP = 1 << 20  # arena task capacity (the largest DAG of this distribution has ~0.87 M tasks)
METRIC = "sim task-events/s (bit-exact)"
UNIT = "task-events/s"
CONFIG = {"workload": "random search, N=65536 Cholesky, b=2048 (32x32 tiles, 5,984 base tasks), split levels "
                      "uniform {0,1,2,3} (finest b=256; DAGs of ~810,000 tasks), 4,096 candidates per launch, all "
                      "resident, simulated on 32 CPU + 2 GPU-type processors (FCFS + EFT-P, transfers, write-back "
                      "caching)",
          "n_tiles": N_TILES, "b": B, "levels": N_LEVELS, "candidates_per_step": N_CAND,
          "platform": "cpu32_gpu2", "seed": SEED, "task_cap": TASK_CAP}

# the 8 x 8-tile random-search step on two platforms (extra key)
C1 = W.WORKLOADS["cfg1"]
C1_PLATS = ("cfg1a", "cfg1b")


def env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


# --------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def free_cuda():
    import gc

    import torch
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


# ---------------------------------------------------------------- GPU arm


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1602_05510_b300 import build, hesp
    from paper_1602_05510_b300.sharding import global_best, rank_first, reduce_timing

    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local = env_int("LOCAL_RANK", 0)
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    n = args.tiles  # 32 (smaller only for profiling)
    cap = args.task_cap
    nb = W.base_count(n)
    C = args.candidates
    plat = hesp.Platform(W.PLATFORMS[PLAT])
    ws = hesp.alloc_workspace(plat, n, MAX_LEVEL, C, cap)  # every candidate resident
    levels = torch.empty(C * nb, dtype=torch.int8, device=dev)
    cands = torch.empty(C * 16, dtype=torch.uint8, device=dev)
    ms = torch.empty(C, dtype=torch.int64, device=dev)
    st = torch.empty(C, dtype=torch.int32, device=dev)
    nt = torch.empty(C, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 126 MB L2
    K = args.steps
    best = torch.empty((max(K, 1), 2), dtype=torch.int64, device=dev)  # per step: (makespan, global index)
    evs = torch.empty((max(K, 1), 2), dtype=torch.int64, device=dev)   # per step: (best, task-events)

    def step(first, k, kev=None):
        # generation, simulation, the batch's best candidate and its task-event count (4 launches)
        hesp.generate_candidates(hesp.GEN_UNIFORM, SEED, first, C, n, B, N_LEVELS, levels, cands)
        if kev is not None:
            kev[0].record(stream)
        hesp.simulate_batch(plat, cands, levels, C, n, MAX_LEVEL, ws, makespan=ms, status=st, ntasks=nt,
                            task_cap=cap)
        if kev is not None:
            kev[1].record(stream)
        hesp.best_candidate(ms, st, first, out=best[k])
        hesp.best_makespan(ms, st, nt, out=evs[k])

    for w in range(args.warmup):
        step(rank_first(rank, world, C, w), 0)
    torch.cuda.synchronize()
    if args.warmup and int((st != 0).sum().item()):
        raise RuntimeError("%d candidates failed" % int((st != 0).sum().item()))

    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    kern_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for k in range(K):
        flush.fill_(k & 0xFF)  # evict L2 between timed steps (outside the step's events)
        step_ev[k][0].record(stream)
        step(rank_first(rank, world, C, args.warmup + k), k, kern_ev[k])
        step_ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    if int((st != 0).sum().item()):
        raise RuntimeError("%d candidates failed" % int((st != 0).sum().item()))
    ev_h = evs[:K].cpu().numpy()
    task_events = int(ev_h[:, 1].sum()) if K else 0
    t_steps = sum(a.elapsed_time(b_) for a, b_ in step_ev) / 1e3
    t_kern = sum(a.elapsed_time(b_) for a, b_ in kern_ev) / 1e3
    t_max, tot_events = reduce_timing(t_steps, task_events, world, dev)
    # the exchange step: every rank's per-step best, combined over ranks
    bests = [global_best(best[k], None, world, dev) for k in range(K)]
    overall = min(bests) if bests else None

    # ---- end to end through the public API with host buffers
    e2e = None
    if args.e2e_steps > 0:
        lv_host = [torch.from_numpy(W.uniform_levels(SEED, rank_first(rank, world, C, 1000 + s), C, nb,
                                                     N_LEVELS).reshape(-1)).pin_memory()
                   for s in range(min(args.e2e_steps, 2))]
        cand_host = hesp.cands_tensor(n, B, np.arange(C, dtype=np.int64) * nb, device="cpu").pin_memory()
        ms_host = torch.empty(C, dtype=torch.int64).pin_memory()
        best_host = torch.empty(2, dtype=torch.int64).pin_memory()
        e2e_ev, e2e_tasks = [], 0
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for s in range(args.e2e_steps):
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(s & 0xFF)
            a.record(stream)
            levels.copy_(lv_host[s % len(lv_host)], non_blocking=True)
            cands.copy_(cand_host, non_blocking=True)
            hesp.simulate_batch(plat, cands, levels, C, n, MAX_LEVEL, ws, makespan=ms, status=st, ntasks=nt,
                                task_cap=cap)
            hesp.best_candidate(ms, st, 0, out=best[0])
            hesp.best_makespan(ms, st, nt, out=evs[0])
            ms_host.copy_(ms, non_blocking=True)
            best_host.copy_(best[0], non_blocking=True)
            b_.record(stream)
            e2e_ev.append((a, b_))
            torch.cuda.synchronize()
            e2e_tasks += int(evs[0, 1].item())
        t_e2e = sum(a.elapsed_time(b_) for a, b_ in e2e_ev) / 1e3
        t_e2e, e2e_tasks = reduce_timing(t_e2e, e2e_tasks, world, dev)
        e2e = {"value": e2e_tasks / t_e2e, "unit": UNIT, "h2d_bytes_per_step": C * nb + C * 16,
               "d2h_bytes_per_step": 8 * C + 16, "steps": args.e2e_steps,
               "path": "pinned host partition vectors -> simulation -> best candidate -> host makespans and best"}
    del ws
    free_cuda()

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    line = {
        "metric": METRIC, "value": tot_events / t_max if t_max > 0 else None, "unit": UNIT,
        "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / max(K, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic (seeded SplitMix64 partition vectors generated on the device)",
        "config": dict(CONFIG, candidates_per_step=C, parallelism="candidates sharded across ranks (dp%d)" % world,
                       l2="256 MB buffer written between timed steps; per-step working set ~220 GB > L2"),
        "profiling_case": None if (n, cap) == (N_TILES, TASK_CAP) else {"n_tiles": n, "task_cap": cap},
        "candidates_per_s": C * world * K / t_max if t_max > 0 else None,
        "task_events": tot_events,
        "wall_s": wall,
        "gpu_launches": 4 * K,  # generation, simulation, best candidate, task-event count
        "kernel_ms_per_step": 1e3 * t_kern / max(K, 1),
        "best_makespan_ns": overall[0] if overall else None,
        "best_candidate": overall[1] if overall else None,
        "clocks": clk,
        "e2e": e2e,
    }
    line["roofline"] = roofline(t_kern / max(K, 1), task_events / max(K, 1), props, peaks, n)
    if world == 1 and (n, cap) == (N_TILES, TASK_CAP):
        extra_clk = ClockSampler(local)
        extra_clk.start()
        if args.extra_cfg1:
            line["random_8x8_two_platforms"] = run_cfg1(args, dev)
            free_cuda()
        if args.search_budget > 0:
            line["search"] = search_comparison(args)
            free_cuda()
        line["extra_clocks"] = extra_clk.stop()
        if args.cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_sample)
            line["cpu_baseline_1core"] = cpu_baseline(args.cpu_sample_1core, threads=1)
    print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_cfg1(args, dev):
    """The 8 x 8-tile random-search step (65,536 candidates, levels uniform
    {0, 1, 2}): generation, largest DAG first, one DAG build launch, then the
    kept DAGs simulated on 12 CPU + 1 GPU-type and on 4 big + 4 LITTLE."""
    import torch

    from paper_1602_05510_b300 import hesp

    n, b, NL, C = C1.n_tiles, C1.b, C1.n_levels, args.cfg1_candidates
    nb = W.base_count(n)
    stream = torch.cuda.current_stream()
    plats = [hesp.Platform(W.PLATFORMS[k]) for k in C1_PLATS]
    kept = hesp.alloc_workspace_kept(n, NL - 1, C)
    levels = torch.empty(C * nb, dtype=torch.int8, device=dev)
    cands = torch.empty(C * 16, dtype=torch.uint8, device=dev)
    scands = torch.empty(C * 16, dtype=torch.uint8, device=dev)
    perm = torch.empty(C, dtype=torch.int32, device=dev)
    sort_ws = hesp.sort_workspace(C, dev)
    bst = torch.empty(C, dtype=torch.int32, device=dev)
    ms = [torch.empty(C, dtype=torch.int64, device=dev) for _ in plats]
    st = [torch.empty(C, dtype=torch.int32, device=dev) for _ in plats]
    nt = [torch.empty(C, dtype=torch.int64, device=dev) for _ in plats]
    tot = torch.empty((len(plats), 2), dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(first):
        hesp.generate_candidates(hesp.GEN_UNIFORM, C1.seed, first, C, n, b, NL, levels, cands)
        sc, _ = hesp.sort_cands_by_size(cands, levels, C, scands, perm, sort_ws)
        hesp.dag_build_kept(sc, levels, C, n, NL - 1, kept, status=bst)
        for i, p in enumerate(plats):
            hesp.simulate_batch_reuse(p, sc, levels, C, n, NL - 1, kept, makespan=ms[i], status=st[i], ntasks=nt[i])

    for w in range(args.cfg1_warmup):
        step(w * C)
    torch.cuda.synchronize()
    K = args.cfg1_steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    events = 0
    for k in range(K):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        step((args.cfg1_warmup + k) * C)
        ev[k][1].record(stream)
        for i in range(len(plats)):
            hesp.best_makespan(ms[i], st[i], nt[i], out=tot[i])
        torch.cuda.synchronize()
        if any(int((s != 0).sum().item()) for s in st):
            raise RuntimeError("8x8-tile candidates failed")
        events += int(tot[:, 1].sum().item())
    t = sum(a.elapsed_time(b_) for a, b_ in ev) / 1e3
    return {"metric": METRIC, "value": events / t, "unit": UNIT, "steps": K, "ms_per_step": 1e3 * t / max(K, 1),
            "candidates_per_s": len(plats) * C * K / t,
            "workload": "random search, N=16384 Cholesky, b=2048 (8x8 tiles, 120 base tasks), split levels uniform "
                        "{0,1,2}, 65,536 candidates per step, largest DAG first, one DAG build launch, simulated on "
                        "12 CPU + 1 GPU-type (transfers, write-back) and on 4 big + 4 LITTLE (shared memory)"}


def run_random8x8(args):
    """The 8 x 8-tile two-platform step on its own line (profiling and
    comparison with the default run's extra key)."""
    import torch

    from paper_1602_05510_b300 import build

    build.build()
    r = run_cfg1(args, torch.device("cuda", 0))
    r.update({"n_gpus": 1, "higher_is_better": True, "candidates_per_step": args.cfg1_candidates})
    print(json.dumps(r))


def search_comparison(args):
    """Best makespan reached on the 32 x 32-tile problem within the same
    wall-time budget by plain batched random search, by surrogate-guided
    search and by the paper's iterative solver (CP selection, Hard sampling,
    from the unsplit partition), one arm after the other on this GPU."""
    from paper_1602_05510_b300 import search as S

    spec = W.PLATFORMS[PLAT]
    ws = int(args.ws_gb * (1 << 30))
    out = {"budget_s": args.search_budget}
    sim = S.Simulator(spec, N_TILES, B, MAX_LEVEL, N_CAND, task_cap=TASK_CAP)
    rlog = S.random_search(spec, N_TILES, B, N_LEVELS, seed=SEED, budget_s=args.search_budget, per_launch=N_CAND,
                           sim=sim)
    del sim
    free_cuda()
    # the surrogate arm starts as the solver does (from the unsplit partition,
    # its descent labelling the model), then ranks mutants of its elites
    scfg = dict(surrogate_cfg(args), start="solver", heldout=1024, p_mut=args.seeded_p_mut)
    slog = S.surrogate_search(spec, N_TILES, B, N_LEVELS, seed=5, budget_s=args.search_budget,
                              per_launch=args.round_sims, cfg=S.SurrogateConfig(**scfg), task_cap=TASK_CAP,
                              ws_bytes=ws)
    free_cuda()
    ilog = S.iterative_search(spec, N_TILES, B, N_LEVELS, S.hesp.SOLVER_CP, S.hesp.PICK_HARD, seed=6,
                              budget_s=args.search_budget, task_cap=TASK_CAP, ws_bytes=ws,
                              first=np.zeros(W.base_count(N_TILES), np.int8))
    target = rlog.best[-1]
    t_reach = slog.time_to_reach(target)
    t_solver = slog.time_to_reach(ilog.best[-1])
    out.update({
        "random": {"best": rlog.best[-1], "candidates": rlog.simulated[-1],
                   "task_events_per_s": rlog.events[-1] / rlog.times[-1]},
        "surrogate": {"best": slog.best[-1], "candidates_simulated": slog.simulated[-1],
                      "start": "the iterative solver's descent from the unsplit partition (CP + Hard), then "
                               "surrogate-ranked mutants of the elites",
                      "time_to_random_best_s": t_reach,
                      "time_ratio": (t_reach / rlog.times[-1]) if t_reach is not None else None,
                      "time_to_solver_best_s": t_solver,
                      "rounds": len(slog.metrics), "last_round": slog.metrics[-1] if slog.metrics else None,
                      "spearman_selected_median": _median([m.get("spearman") for m in slog.metrics]),
                      "spearman_heldout_median": _median([m.get("heldout_spearman") for m in slog.metrics])},
        "iterative_cp_hard": {"best": ilog.best[-1], "candidates_simulated": ilog.simulated[-1],
                              "iterations": len(ilog.best), "time_to_random_best_s": ilog.time_to_reach(target),
                              "first_local_optimum": ilog.metrics[0] if ilog.metrics else None},
    })
    return out


def _median(xs):
    xs = [x for x in xs if x is not None and np.isfinite(x)]
    return float(np.median(xs)) if xs else None


def surrogate_cfg(args):
    return dict(hidden=512, batch=2048, warmup_launches=1, warmup_steps=args.warmup_steps,
                steps_per_round=args.round_steps, proposals=args.round_proposals, elites=32, p_mut=args.p_mut,
                label_cap=1 << 17)


# ncu figures of the simulation kernel taken on the kernel source whose sha1
# prefix is given (null once the source changes): DRAM bytes and issued
# warp-instructions per task-event and the share of issue slots busy.
SIM_NCU = {"source_sha1_12": "625d145ba2bb",
           # one 1-pass capture of a full 4,096-candidate launch: 1.05 TB read + 0.5756 TB written
           "dram_bytes_per_task_event": (1.05e12 + 0.5756e12) / 3316708562,
           # --set full on a 10x10-tile launch of the same kernel (3,072 candidates)
           "warp_inst_per_task_event": 54.446167e9 / 78173006, "issue_active_pct": 49.34, "warps_per_sm": 18.09,
           "case": "DRAM bytes: the full 4,096-candidate launch (one pass); instructions and issue slots: a "
                   "10x10-tile launch of 3,072 candidates (20.8 warps per SM)"}


def sim_source_matches():
    p = os.path.join(ROOT, "paper_1602_05510_b300", "csrc", "sim_kernel.cu")
    try:
        return hashlib.sha1(open(p, "rb").read()).hexdigest()[:12] == SIM_NCU["source_sha1_12"]
    except OSError:
        return False


def roofline(t, events, props, peaks, n=N_TILES):
    """Dominant kernel: the simulation launch (expansion, dependences and the
    event loop of every candidate).  It is bound by integer and control
    issue, not by HBM or tensor cores.  `achieved` counts the algorithmic
    int64 operations per task-event (EFT evaluation 4 P, data-ready times
    M A_j, coherence commit A_j) over one launch's task-events, divided by the
    launch's CUDA-event time; the peak is the SM integer issue rate at the
    maximum SM clock (SMs x 128 INT32 lanes, one int64 operation = 2
    lane-operations).  Beside it: the issue-slot view (warp-instructions per
    task-event from ncu, times the live task-event rate, against SMs x 4
    schedulers x clock)."""
    spec = W.PLATFORMS[PLAT]
    alg = alg_ops_per_event(W.uniform_levels(SEED, 0, 256, W.base_count(n), N_LEVELS), n, B,
                            len(spec.procs), spec.n_mem)
    sm_max = (peaks or {}).get("sm_max_mhz", 2032.0)
    sms = props.multi_processor_count
    peak = sms * 128 * sm_max * 1e6 / 2 / 1e12  # T int64-op/s
    achieved = alg * events / t / 1e12 if t > 0 and alg else None
    fresh = sim_source_matches()
    issue_peak = sms * 4 * sm_max * 1e6
    ipe = SIM_NCU["warp_inst_per_task_event"] if fresh else None
    out = {"bound": "alu", "kernel": "sim_kernel<M=3,NS=2> (cpu32_gpu2; 72 registers, 4-warp CTAs)", "achieved": achieved, "peak": peak,
           "unit": "T int64-op/s", "frac": achieved / peak if achieved else None,
           "peak_source": "derived: %d SMs x 128 INT32 lanes x %.0f MHz / 2 (sm_max_mhz of MEASURED_PEAKS)"
                          % (sms, sm_max),
           "kernel_ms": 1e3 * t, "task_events_per_launch": events, "alg_ops_per_task_event": alg,
           "traffic": SIM_NCU["dram_bytes_per_task_event"] * events if fresh else None,
           "dram_gbs": SIM_NCU["dram_bytes_per_task_event"] * events / t / 1e9 if fresh and t > 0 else None,
           "traffic_note": "DRAM bytes per task-event from ncu (%s), times this launch's task-events; "
                           "algorithmic I/O is 5,984 B in + 24 B out per candidate" % SIM_NCU["case"],
           "issue_slots": {"warp_inst_per_task_event": ipe,
                           "achieved_frac_of_issue_peak": ipe * events / t / issue_peak if ipe and t > 0 else None,
                           "issue_peak_warp_inst_per_s": issue_peak,
                           "ncu_issue_active_pct": SIM_NCU["issue_active_pct"] if fresh else None,
                           "ncu_warps_per_sm": SIM_NCU["warps_per_sm"] if fresh else None,
                           "source": "ncu smsp__inst_executed.sum / task-events, "
                                     "smsp__issue_active.avg.pct_of_peak_sustained_active"}}
    return out


def alg_ops_per_event(levels, n, b, P, M):
    """Algorithmic int64 operations per task-event of one launch: 4 P for the
    EFT evaluation (two max, one add, one compare per processor) plus
    (M + 1) per atom of the task's data (data-ready time per memory, then the
    coherence commit), with atoms of side b >> (candidate's deepest level)."""
    from paper_1602_05510_b300 import hesp
    kids = {0: (2, 1, 1, 0), 1: (0, 4, 0, 2), 2: (0, 0, 4, 2), 3: (0, 0, 0, 8)}
    nreg = np.array([1, 2, 2, 3])
    tab = np.zeros((4, 5, 4), np.int64)
    for op in range(4):
        tab[op, 0, op] = 1
    for l in range(1, 5):
        for op in range(4):
            tab[op, l] = sum(kids[op][c] * tab[c, l - 1] for c in range(4))
    lv = np.asarray(levels, np.int64)
    ops = hesp.Dag(n, b, int(lv.max())).base_tasks()[0]
    Lc = lv.max(axis=1, keepdims=True)
    tasks = tab[ops[None, :], lv].sum(-1)                  # [C, n_base]
    regs = (tab[ops[None, :], lv] * nreg).sum(-1)
    atoms = regs * (4 ** (Lc - lv))
    return 4 * P + (M + 1) * atoms.sum() / tasks.sum()


def cpu_baseline(sample, threads=None):
    """The oracle on `sample` candidates of the same workload, one candidate
    per thread chunk over the host cores (or `threads`)."""
    import oracle as O

    cores = threads or os.cpu_count() or 1
    lv = W.uniform_levels(SEED, 0, sample, W.base_count(N_TILES), N_LEVELS)
    pl = O.make_platform(W.PLATFORMS[PLAT])
    t0 = time.perf_counter()
    ms, st, tasks = O.simulate_many(pl, N_TILES, B, lv, threads=cores)
    dt = time.perf_counter() - t0
    assert (st == 0).all()
    ev = int(tasks.sum())
    return {"value": ev / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "candidates_per_s": sample / dt,
            "sample": "%d candidates of the same workload (%d task-events) on %d host thread(s), %.1f s; per "
                      "task-event rate, so it extrapolates to a 4,096-candidate launch" % (sample, ev, cores, dt)}


def cpu_baseline_each(sim_one, count, label):
    """The oracle timed on the host cores over `count` candidates of a
    general-path workload: sim_one(c) simulates candidate c and returns its
    task count (ctypes releases the GIL, so Python threads run in parallel)."""
    from concurrent.futures import ThreadPoolExecutor

    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        ev = sum(ex.map(sim_one, range(count)))
    dt = time.perf_counter() - t0
    return {"value": ev / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d candidates of the same workload (%s, %d task-events) over %d host threads, %.1f s"
                      % (count, label, ev, cores, dt)}


# ---------------------------------------------------------- reference arm


def run_reference(args):
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    if rank != 0:
        return
    import oracle as O

    O.build()
    cores = os.cpu_count() or 1
    per_step = args.ref_sample or cores  # one candidate per host thread per step
    pl = O.make_platform(W.PLATFORMS[PLAT])
    nb = W.base_count(N_TILES)

    def one(k):
        lv = W.uniform_levels(SEED, k * per_step, per_step, nb, N_LEVELS)
        _, st, tasks = O.simulate_many(pl, N_TILES, B, lv, threads=cores)
        assert (st == 0).all()
        return int(tasks.sum())

    for w in range(args.warmup):
        one(w)
    t0 = time.perf_counter()
    ev = 0
    for k in range(args.steps):
        ev += one(args.warmup + k)
    dt = time.perf_counter() - t0
    v = ev / dt
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic", "impl": "reference",
            "config": dict(CONFIG, parallelism="host threads"),
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": v, "unit": UNIT,
                             "sample": "%d candidates of the same workload per step on %d host threads"
                                       % (per_step, cores)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------- other workload lines


def run_surrogate_pipeline(args):
    """16 x 16 tiles (816 base tasks, levels 0..2) on 16 CPU + 2 GPU-type
    processors: label n_labels uniform partitions by exact simulation, train
    the 2448 -> 512 -> 512 -> 1 surrogate on them, rank 4M proposals, re-simulate
    the best 1 % exactly and report the surrogate's relative makespan error
    and Spearman rank correlation on that slice, with the throughput of each
    stage."""
    import torch

    from paper_1602_05510_b300 import build, hesp
    from paper_1602_05510_b300 import search as S

    build.build()
    n, b, NL = 16, 2048, 3
    nb = W.base_count(n)
    spec = W.PLATFORMS["cfg3"]
    N = args.labels
    P = args.proposals
    K = P // 100
    sim = S.Simulator(spec, n, b, NL - 1, min(N, 65536))
    lab_lv = torch.empty(N * nb, dtype=torch.int8, device="cuda")
    lab_ms = torch.empty(N, dtype=torch.int64, device="cuda")
    ev = 0

    def sync():
        torch.cuda.synchronize()
        return time.perf_counter()

    t0 = sync()
    for i in range(0, N, sim.per_launch):
        c = min(sim.per_launch, N - i)
        hesp.generate_candidates(hesp.GEN_UNIFORM, 3, i, c, n, b, NL, lab_lv[i * nb:])
        ms, st, nt = sim.run(lab_lv[i * nb:], c)
        lab_ms[i:i + c].copy_(ms)
        ev += int(hesp.best_makespan(ms, st, nt).cpu().numpy()[1])
    t_label = sync() - t0
    sur = hesp.Surrogate(nb, NL, 512, 65536, seed=3)  # inference in chunks of 65,536 rows
    sur.fit_stats(lab_ms)
    mu, sigma, _ = sur.stats()
    t0 = sync()
    losses = torch.empty(args.train_steps, dtype=torch.float32, device="cuda")
    sur.train(lab_lv, lab_ms, N, 4096, args.train_steps, 1e-3, seed=7, loss=losses)
    t_train = sync() - t0
    prop = torch.empty(P * nb, dtype=torch.int8, device="cuda")
    hesp.generate_candidates(hesp.GEN_UNIFORM, 33, 0, P, n, b, NL, prop)
    pred = torch.empty(P, dtype=torch.float32, device="cuda")
    sur.infer(prop, min(P, 65536), pred)  # warm-up
    t0 = sync()
    sur.infer(prop, P, pred)
    idx = hesp.select_topk(pred, K)
    t_infer = sync() - t0
    cands = hesp.make_cands(idx, n, b)
    sim2 = S.Simulator(spec, n, b, NL - 1, K)
    t0 = sync()
    ms, st, nt = sim2.run(prop, K, cands)
    t_resim = sync() - t0
    rel, rho = hesp.rank_metrics(hesp.gather_f32(pred, idx), ms, mu, sigma)
    flops = 2.0 * P * (sur.Fp * 512 + 512 * 512 + 512)
    L = losses.cpu().numpy()
    line = {"metric": "surrogate proposals ranked/s (2448-512-512-1 bf16 MLP + top-1% select)",
            "value": P / t_infer, "unit": "proposals/s", "n_gpus": 1, "higher_is_better": True,
            "workload": "16x16 tiles, levels 0..2, 16 CPU + 2 GPU; %d labels, %d proposals, top %d" % (N, P, K),
            "labelling_task_events_per_s": ev / t_label, "label_s": t_label,
            "train_steps": args.train_steps, "train_step_ms": 1e3 * t_train / max(args.train_steps, 1),
            "train_loss_first_last": [float(L[:10].mean()), float(L[-10:].mean())],
            "infer_tflops": flops / t_infer / 1e12, "resim_s": t_resim,
            "top1pct_rel_makespan_error": rel, "top1pct_spearman": rho, "mu": mu, "sigma": sigma,
            "error_flag": sur.error_flag()}
    print(json.dumps(line))


def run_uneven(args):
    """Ragged batch: 16,384 candidates per launch with n in [4, 32] tiles,
    b in {512, 1024, 2048}, levels {0: .5, 1: .3, 2: .2} on 16 CPU + 2 GPU-type
    processors; the launch shape is autotuned on a sample, then
    generation + simulation is captured once as a CUDA graph and replayed."""
    import torch

    from paper_1602_05510_b300 import build, hesp

    build.build()
    C = 16384
    spec = W.PLATFORMS["cfg2"]
    plat = hesp.Platform(spec)
    cap = 100000  # the largest DAG of this distribution has 88,272 tasks
    ws = hesp.alloc_workspace(plat, 32, 2, C, task_cap=cap)
    s = torch.cuda.Stream()
    cands = torch.empty(C * 16, dtype=torch.uint8, device="cuda")
    lcap = C * W.base_count(32)
    levels = torch.empty(lcap, dtype=torch.int8, device="cuda")
    used = torch.zeros(1, dtype=torch.int64, device="cuda")
    ms = torch.empty(C, dtype=torch.int64, device="cuda")
    st = torch.empty(C, dtype=torch.int32, device="cuda")
    nt = torch.empty(C, dtype=torch.int64, device="cuda")
    sorted_c = torch.empty(C * 16, dtype=torch.uint8, device="cuda")
    perm = torch.empty(C, dtype=torch.int32, device="cuda")
    sort_ws = torch.empty((65536 + C) * 4, dtype=torch.uint8, device="cuda")
    hesp.generate_uneven(2, 0, C, cands, levels, used, stream=s)
    hesp.sort_cands_by_size(cands, levels, C, sorted_c, perm, sort_ws, stream=s)
    s.synchronize()
    (tc, tb), times = hesp.autotune(plat, sorted_c, levels, C, 32, 2, ws, task_cap=cap, stream=s)

    def step():
        # generate, order largest first, simulate (results in sorted order; perm maps back)
        hesp.generate_uneven(2, 0, C, cands, levels, used, stream=s)
        hesp.sort_cands_by_size(cands, levels, C, sorted_c, perm, sort_ws, stream=s)
        hesp.simulate_batch(plat, sorted_c, levels, C, 32, 2, ws, makespan=ms, status=st, ntasks=nt, task_cap=cap,
                            stream=s)

    step()
    s.synchronize()
    g = hesp.Graph.capture(s, step)
    for _ in range(args.warmup):
        g.launch(s)
    s.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b_ in ev:
        a.record(s)
        g.launch(s)
        b_.record(s)
    s.synchronize()
    t = sum(a.elapsed_time(b_) for a, b_ in ev) / 1e3
    ok = int((st == 0).sum().item())
    tasks = int(nt[st == 0].sum().item())
    line = {"metric": "sim task-events/s (bit-exact)", "value": tasks * args.steps / t, "unit": "task-events/s",
            "n_gpus": 1, "steps": args.steps, "higher_is_better": True,
            "workload": "ragged batch of 16,384 candidates (n 4..32 tiles, b 512..2048, levels .5/.3/.2), "
                        "16 CPU + 2 GPU-type processors, largest-first order, CUDA-graph replay",
            "ms_per_launch": 1e3 * t / args.steps, "candidates_ok": ok, "task_events_per_launch": tasks,
            "autotuned": {"ctas_per_sm": tc, "bitmap": "global" if tb == 1 else "shared", "ms_by_shape": times}}
    print(json.dumps(line))


def run_factors(args):
    """General partition parameter (one-level k-way partitions, p = 1/k):
    65,536 candidates of 8 x 8 tiles of b = 3072 with factors uniform in
    {1, 2, 3, 4} (non-dyadic tilings wherever 3 meets 2 or 4), simulated on
    both platforms of the default workload; inputs resident on the device, a
    256 MB buffer written between steps."""
    import torch

    from paper_1602_05510_b300 import build, hesp

    build.build()
    n, b, K = W.FACTOR_N, W.FACTOR_B, W.FACTOR_MAX
    C = args.general_candidates
    nb = W.base_count(n)
    f = torch.from_numpy(W.uniform_factors(9, 0, C, nb, K).reshape(-1).copy()).cuda()
    cands = hesp.cands_tensor(n, b, np.arange(C, dtype=np.int64) * nb)
    plats = [hesp.Platform(W.PLATFORMS[k]) for k in C1_PLATS]
    wss = [hesp.alloc_workspace_factors(p, n, K, C) for p in plats]
    ms = [torch.empty(C, dtype=torch.int64, device="cuda") for _ in plats]
    st = [torch.empty(C, dtype=torch.int32, device="cuda") for _ in plats]
    nt = [torch.empty(C, dtype=torch.int64, device="cuda") for _ in plats]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        for i, p in enumerate(plats):
            hesp.simulate_factors(p, cands, f, C, n, K, b, wss[i], makespan=ms[i], status=st[i], ntasks=nt[i])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    t_k = [0.0 for _ in plats]
    for it in range(args.steps):
        flush.fill_(it & 255)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(plats) + 1)]
        ev[0].record()
        for i, p in enumerate(plats):
            hesp.simulate_factors(p, cands, f, C, n, K, b, wss[i], makespan=ms[i], status=st[i], ntasks=nt[i])
            ev[i + 1].record()
        torch.cuda.synchronize()
        for i in range(len(plats)):
            t_k[i] += ev[i].elapsed_time(ev[i + 1]) / 1e3
    ok = all(bool((x == 0).all().item()) for x in st)
    events = sum(int(x.sum().item()) for x in nt)
    t = sum(t_k)
    line = {"metric": METRIC, "value": events * args.steps / t, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "int64", "data": "synthetic",
            "workload": "non-dyadic partitions: N=24576 Cholesky, b=3072 (8x8 tiles, 120 base tasks), one "
                        "partition factor k in {1,2,3,4} (p = 1/k) per base task, %d candidates, atoms of "
                        "b / lcm(factors), simulated on 12 CPU + 1 GPU-type and on 4 big + 4 LITTLE" % C,
            "ms_per_step": 1e3 * t / args.steps, "all_ok": ok, "task_events_per_step": events,
            "candidates_per_s": C * len(plats) * args.steps / t,
            "kernel_ms_per_step": {k: 1e3 * x / args.steps for k, x in zip(C1_PLATS, t_k)},
            "l2": "256 MB buffer written between timed steps"}
    if args.cpu_baseline:
        import oracle as O

        fh = W.uniform_factors(9, 0, 8192, nb, K)
        pls = [O.make_platform(W.PLATFORMS[k]) for k in C1_PLATS]

        def one(c):
            return sum(O.simulate_factors(pl, n, b, fh[c], schedule=False)["n_tasks"] for pl in pls)

        line["cpu_baseline"] = cpu_baseline_each(one, 8192, "both platforms")
    print(json.dumps(line))


def run_capacity(args):
    """Finite accelerator memories: the default workload's 65,536 candidates
    (8 x 8 tiles, b = 2048, levels {0, 1, 2}) on 12 CPU + 1 GPU-type
    processor whose memory holds 256 MB (8 tiles of the 64 the matrix
    needs): LRU eviction with write-back, simulated exactly."""
    import torch

    from paper_1602_05510_b300 import build, hesp

    build.build()
    C = args.general_candidates
    n1, b1, nl1, ml1 = C1.n_tiles, C1.b, C1.n_levels, C1.n_levels - 1
    nb = W.base_count(n1)
    plat = hesp.Platform(W.PLATFORMS["cfg1a"], capacity={1: 256 << 20})
    cands = torch.empty(C * 16, dtype=torch.uint8, device="cuda")
    levels = torch.empty(C * nb, dtype=torch.int8, device="cuda")
    hesp.generate_candidates(hesp.GEN_UNIFORM, C1.seed, 0, C, n1, b1, nl1, levels, cands)
    ws = hesp.alloc_workspace(plat, n1, ml1, C)
    ms = torch.empty(C, dtype=torch.int64, device="cuda")
    st = torch.empty(C, dtype=torch.int32, device="cuda")
    nt = torch.empty(C, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        hesp.simulate_batch(plat, cands, levels, C, n1, ml1, ws, makespan=ms, status=st, ntasks=nt)
    torch.cuda.synchronize()
    t = 0.0
    for it in range(args.steps):
        flush.fill_(it & 255)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        hesp.simulate_batch(plat, cands, levels, C, n1, ml1, ws, makespan=ms, status=st, ntasks=nt)
        e.record()
        torch.cuda.synchronize()
        t += a.elapsed_time(e) / 1e3
    events = int(nt.sum().item())
    line = {"metric": METRIC, "value": events * args.steps / t, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "int64", "data": "synthetic",
            "workload": "finite GPU memory: N=16384 Cholesky, b=2048 (8x8 tiles), levels uniform {0,1,2}, "
                        "%d candidates on 12 CPU + 1 GPU-type with 256 MB of GPU memory (LRU eviction, "
                        "write-back)" % C,
            "ms_per_step": 1e3 * t / args.steps, "all_ok": bool((st == 0).all().item()),
            "task_events_per_step": events, "candidates_per_s": C * args.steps / t,
            "mean_makespan_ns": float(ms.double().mean().item()), "l2": "256 MB buffer written between timed steps"}
    if args.cpu_baseline:
        import oracle as O

        lh = W.workload_levels("cfg1", 0, 8192)
        pl = O.make_platform(W.PLATFORMS["cfg1a"], capacity={1: 256 << 20})

        def one(c):
            return O.simulate(pl, n1, b1, lh[c], schedule=False)["n_tasks"]

        line["cpu_baseline"] = cpu_baseline_each(one, 8192, "12 CPU + 1 GPU-type, 256 MB GPU memory")
    print(json.dumps(line))


def run_exhaustive(args):
    """The exhaustive search of the 3 x 3-tile problem (N = 3072, b = 1024):
    all 1,024 partitions (each base task split once or not), generated,
    simulated on 4 CPU + 1 GPU-type processors and reduced to the best
    makespan on the device, captured as one CUDA graph and replayed; the
    oracle runs the same search on the host cores."""
    import torch

    import oracle as O
    from paper_1602_05510_b300 import build, hesp

    build.build()
    C, n, b, L = 1024, 3, 1024, 1
    spec = W.PLATFORMS["cfg0"]
    plat = hesp.Platform(spec)
    ws = hesp.alloc_workspace(plat, n, L, C)
    s = torch.cuda.Stream()
    levels = torch.empty(C * 10, dtype=torch.int8, device="cuda")
    cands = torch.empty(C * 16, dtype=torch.uint8, device="cuda")
    ms = torch.empty(C, dtype=torch.int64, device="cuda")
    st = torch.empty(C, dtype=torch.int32, device="cuda")
    nt = torch.empty(C, dtype=torch.int64, device="cuda")
    best = torch.empty(2, dtype=torch.int64, device="cuda")
    R = 50  # exhaustive searches per graph

    def step():
        for _ in range(R):
            hesp.generate_candidates(hesp.GEN_EXHAUSTIVE, 0, 0, C, n, b, 2, levels, cands, stream=s)
            hesp.simulate_batch(plat, cands, levels, C, n, L, ws, makespan=ms, status=st, ntasks=nt, stream=s)
            hesp.best_makespan(ms, st, nt, out=best, stream=s)

    step()
    s.synchronize()
    g = hesp.Graph.capture(s, step)
    for _ in range(max(args.warmup, 3)):
        g.launch(s)
    s.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b_ in ev:
        a.record(s)
        g.launch(s)
        b_.record(s)
    s.synchronize()
    t = sum(a.elapsed_time(b_) for a, b_ in ev) / 1e3
    searches = R * args.steps
    tasks = int(nt.sum().item())
    best_ms, _ = (int(x) for x in best.cpu().numpy())
    lv_host = W.exhaustive_levels(10)
    pl = O.make_platform(spec)
    t0 = time.perf_counter()
    oms, ost, otasks = O.simulate_many(pl, n, b, lv_host, threads=os.cpu_count() or 1)
    t_cpu = time.perf_counter() - t0
    assert (ost == 0).all() and int(oms.min()) == best_ms
    line = {"metric": "sim task-events/s (bit-exact)", "value": tasks * searches / t, "unit": "task-events/s",
            "n_gpus": 1, "steps": args.steps, "higher_is_better": True,
            "workload": "exhaustive search, N=3072, b=1024 (3x3 tiles, 10 base tasks split once or not: 1,024 "
                        "partitions, %d task-events), 4 CPU + 1 GPU-type processors; %d searches per CUDA graph"
                        % (tasks, R),
            "us_per_search": 1e6 * t / searches, "best_makespan": best_ms,
            "best_partition_count": int((oms == best_ms).sum()),
            "cpu_baseline": {"value": int(otasks.sum()) / t_cpu, "unit": "task-events/s", "cores": os.cpu_count(),
                             "kind": "oracle", "us_per_search": 1e6 * t_cpu}}
    print(json.dumps(line))


def run_search(args):
    """32 x 32 tiles (5984 base tasks, levels 0..3) on 32 CPU + 2 GPU-type
    processors, each arm for the same wall-time budget on one GPU: plain
    batched random search; surrogate-guided search started from the
    iterative solver's descent; the same without the model (mutants of the
    same elites simulated unranked: the ablation); surrogate-guided search
    started from uniform random launches; the paper's iterative solver (CP
    selection, Hard sampling) from the unsplit partition."""
    from paper_1602_05510_b300 import build, hesp
    from paper_1602_05510_b300 import search as S

    build.build()
    n, b, NL = N_TILES, B, N_LEVELS
    spec = W.PLATFORMS[PLAT]
    ws = int(args.ws_gb * (1 << 30))
    sim = S.Simulator(spec, n, b, NL - 1, args.per_launch, task_cap=TASK_CAP)
    rlog = S.random_search(spec, n, b, NL, seed=SEED, budget_s=args.budget, per_launch=args.per_launch, sim=sim)
    del sim
    free_cuda()
    base = surrogate_cfg(args)
    arms = {}
    for name, extra in (("surrogate_solver_start", dict(start="solver", heldout=1024, p_mut=args.seeded_p_mut)),
                        ("mutation_without_surrogate_solver_start",
                         dict(start="solver", p_mut=args.seeded_p_mut, use_surrogate=False)),
                        ("surrogate_random_start", dict(heldout=1024))):
        lg = S.surrogate_search(spec, n, b, NL, seed=5, budget_s=args.budget, per_launch=args.round_sims,
                                cfg=S.SurrogateConfig(**dict(base, **extra)), task_cap=TASK_CAP, ws_bytes=ws)
        arms[name] = lg
        free_cuda()
    ilog = S.iterative_search(spec, n, b, NL, hesp.SOLVER_CP, hesp.PICK_HARD, seed=6, budget_s=args.budget,
                              task_cap=TASK_CAP, ws_bytes=ws, first=np.zeros(W.base_count(n), np.int8))
    target = rlog.best[-1]
    line = {"metric": "best makespan in %.0f s, surrogate vs plain search" % args.budget, "unit": "ns",
            "higher_is_better": False, "n_gpus": 1,
            "workload": "32x32 tiles, b=2048, levels 0..3, 32 CPU + 2 GPU-type processors",
            "random": {"best": rlog.best[-1], "candidates": rlog.simulated[-1], "task_events": rlog.events[-1],
                       "task_events_per_s": rlog.events[-1] / rlog.times[-1],
                       "trace": list(zip(rlog.times, rlog.best))},
            "iterative_cp_hard": {"best": ilog.best[-1], "candidates_simulated": ilog.simulated[-1],
                                  "iterations": len(ilog.best), "task_events": ilog.events[-1],
                                  "trace": list(zip(ilog.times, ilog.best)), "restarts": ilog.metrics,
                                  "time_to_random_best_s": ilog.time_to_reach(target)}}
    for name, lg in arms.items():
        t_reach = lg.time_to_reach(target)
        line[name] = {"best": lg.best[-1], "candidates_simulated": lg.simulated[-1], "task_events": lg.events[-1],
                      "time_to_random_best_s": t_reach,
                      "time_ratio": (t_reach / rlog.times[-1]) if t_reach is not None else None,
                      "time_to_solver_best_s": lg.time_to_reach(ilog.best[-1]),
                      "spearman_selected_median": _median([m.get("spearman") for m in lg.metrics]),
                      "spearman_heldout_median": _median([m.get("heldout_spearman") for m in lg.metrics]),
                      "rel_err_heldout_median": _median([m.get("heldout_rel_err") for m in lg.metrics]),
                      "rounds": len(lg.metrics), "trace": list(zip(lg.times, lg.best))}
    print(json.dumps(line))


def run_solver(args):
    """HeSP's iterative solver (Sec. 2.1) with each selection policy (All, CP,
    Shallow) and sampling type (Hard, Soft) on 8 x 8 tiles (120 base tasks,
    levels 0..2, 12 CPU + 1 GPU-type processors), starting from the unsplit
    partition and restarting from uniform random ones at each local optimum,
    next to plain batched random search, each for the same wall time."""
    import torch

    from paper_1602_05510_b300 import build, hesp
    from paper_1602_05510_b300 import search as S

    build.build()
    n, b, NL = 8, 2048, 3
    spec = W.PLATFORMS["cfg1a"]
    B = args.solver_budget
    arms = {}
    rlog = S.random_search(spec, n, b, NL, seed=4, budget_s=B, per_launch=4096)
    arms["random"] = {"best": rlog.best[-1], "candidates_simulated": rlog.simulated[-1],
                      "task_events": rlog.events[-1]}
    for mode, mname in ((hesp.SOLVER_ALL, "all"), (hesp.SOLVER_CP, "cp"), (hesp.SOLVER_SHALLOW, "shallow")):
        for pick, pname in ((hesp.PICK_HARD, "hard"), (hesp.PICK_SOFT, "soft")):
            lg = S.iterative_search(spec, n, b, NL, mode, pick, seed=6, budget_s=B, first=np.zeros(120, np.int8))
            first_opt = lg.metrics[0] if lg.metrics else None
            arms["%s_%s" % (mname, pname)] = {
                "best": lg.best[-1], "candidates_simulated": lg.simulated[-1], "task_events": lg.events[-1],
                "iterations": len(lg.best), "restarts": len(lg.metrics),
                "first_local_optimum": first_opt,
                "time_to_random_best_s": lg.time_to_reach(rlog.best[-1])}
            torch.cuda.synchronize()
    # the solver over partition factors (p = 1/k, k in 1..4) on 8 x 8 tiles of 3072
    fb = W.FACTOR_B
    for mode, mname in ((hesp.SOLVER_ALL, "all"), (hesp.SOLVER_CP, "cp")):
        sv = S.IterativeSolver(spec, n, fb, W.FACTOR_MAX, mode, hesp.PICK_HARD, factors=True)
        lg = S.iterative_search(spec, n, fb, W.FACTOR_MAX, mode, hesp.PICK_HARD, seed=6, budget_s=B, solver=sv,
                                first=np.ones(120, np.int8))
        arms["factors_%s_hard" % mname] = {
            "best": lg.best[-1], "candidates_simulated": lg.simulated[-1], "task_events": lg.events[-1],
            "iterations": len(lg.best), "restarts": len(lg.metrics),
            "first_local_optimum": lg.metrics[0] if lg.metrics else None,
            "best_after_first_iteration": lg.best[0] if lg.best else None}
        torch.cuda.synchronize()
    line = {"metric": "best makespan in %.0f s per arm, iterative solver policies vs plain search" % B,
            "unit": "ns", "higher_is_better": False, "n_gpus": 1,
            "workload": "8x8 tiles, b=2048, levels 0..2, 12 CPU + 1 GPU-type processors; solver arms start "
                        "from the unsplit partition; factors_* arms: the solver over partition factors "
                        "k in 1..4 (p = 1/k) on 8x8 tiles of b=3072", "arms": arms}
    print(json.dumps(line))


def run_table1(args):
    """The paper's Table 1 procedure on the synthetic cost model, for a
    CPU-GPU machine shaped like its 28-core + 3-GPU one (N = 32768, single
    precision transfers) and a 4 big + 4 LITTLE one (N = 8192): per
    scheduling policy, the best homogeneous tile size and the heterogeneous
    partition the All/Soft iterative solver reaches from it."""
    import dataclasses

    from paper_1602_05510_b300 import build
    from paper_1602_05510_b300 import table1 as TB

    build.build()
    plats = [("cpu28_gpu3 (N=32768, fp32)",
              dataclasses.replace(W.cpu_gpu_platform(28, 3), bytes_per_elem=4), 32768, (512, 1024, 2048, 4096)),
             ("big4_little4 (N=8192, fp64)", W.big_little_platform(), 8192, (128, 256, 512, 1024, 2048))]
    out = {}
    for pname, spec, N, sizes in plats:
        rows = []
        for name, order, select in TB.POLICIES:
            t0 = time.perf_counter()
            r = TB.table_row(spec, N, sizes, order, select, rp_seed=1, max_level=3, iterations=args.table_iters,
                             seed=2, task_cap=1 << 20, ws_bytes=48 << 30)
            rows.append({"policy": name, "homog_gflops": r["homog"]["gflops"],
                         "homog_load_pct": 100 * r["homog"]["load"], "homog_block": r["homog_block"],
                         "het_gflops": r["het"]["gflops"], "improvement_pct": r["improvement"],
                         "het_load_pct": 100 * r["het"]["load"], "avg_block": r["het"]["avg_block"],
                         "dag_depth": r["het"]["depth"], "solver_iterations": r["iterations"],
                         "sweep_makespans": r["sweep"], "s": time.perf_counter() - t0})
        out[pname] = rows
    print(json.dumps({"metric": "Table 1 procedure (homogeneous sweep + All/Soft iterative solver)", "n_gpus": 1,
                      "cost_model": "synthetic (CPU 30 GFLOP/s h=96, GPU 2500 GFLOP/s h=768, big 12, LITTLE 3)",
                      "tables": out}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hesp", choices=["hesp", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-sample", type=int, default=64, help="oracle candidates timed on all host cores")
    ap.add_argument("--cpu-sample-1core", type=int, default=12, help="oracle candidates timed on one host core")
    ap.add_argument("--ref-sample", type=int, default=0, help="reference arm: candidates per step (0: one per core)")
    ap.add_argument("--candidates", type=int, default=N_CAND,
                    help="candidates per step (default: the workload's 4,096; smaller only for profiling)")
    ap.add_argument("--tiles", type=int, default=N_TILES,
                    help="tiles per matrix side (default 32; smaller only for profiling captures)")
    ap.add_argument("--task-cap", type=int, default=TASK_CAP, help="arena task capacity (profiling captures)")
    ap.add_argument("--no-extra-cfg1", dest="extra_cfg1", action="store_false",
                    help="skip the 8x8-tile two-platform line of the default run")
    ap.add_argument("--cfg1-steps", type=int, default=5)
    ap.add_argument("--cfg1-candidates", type=int, default=C1.n_cand,
                    help="candidates of the 8x8-tile step (default 65,536; smaller only for profiling)")
    ap.add_argument("--cfg1-warmup", type=int, default=3)
    ap.add_argument("--search-budget", type=float, default=60.0,
                    help="seconds per arm of the search comparison of the default run (0: skip)")
    ap.add_argument("--general-candidates", type=int, default=65536,
                    help="candidates per launch of the factors / capacity workloads")
    ap.add_argument("--workload", default="random", choices=["random", "random8x8", "surrogate", "search", "uneven",
                                                            "solver", "table1", "exhaustive", "factors", "capacity"],
                    help="random: the default benchmark line; surrogate: label/train/rank/re-score "
                         "pipeline; search: surrogate-guided vs random search with the ablation arm")
    ap.add_argument("--labels", type=int, default=1 << 20)
    ap.add_argument("--proposals", type=int, default=1 << 22)
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--budget", type=float, default=60.0)
    ap.add_argument("--solver-budget", type=float, default=10.0)
    ap.add_argument("--table-iters", type=int, default=40)
    ap.add_argument("--per-launch", type=int, default=4096)
    ap.add_argument("--round-sims", type=int, default=1024)
    ap.add_argument("--round-proposals", type=int, default=65536)
    ap.add_argument("--round-steps", type=int, default=40)
    ap.add_argument("--warmup-steps", type=int, default=200)
    ap.add_argument("--p-mut", type=float, default=0.004)
    ap.add_argument("--seeded-p-mut", type=float, default=0.001,
                    help="mutation rate of the solver-seeded surrogate arm of the default run")
    ap.add_argument("--ws-gb", type=float, default=100.0)
    args = ap.parse_args()
    if args.workload == "random8x8":
        return run_random8x8(args)
    if args.workload == "surrogate":
        return run_surrogate_pipeline(args)
    if args.workload == "search":
        return run_search(args)
    if args.workload == "uneven":
        return run_uneven(args)
    if args.workload == "solver":
        return run_solver(args)
    if args.workload == "table1":
        return run_table1(args)
    if args.workload == "capacity":
        return run_capacity(args)
    if args.workload == "factors":
        return run_factors(args)
    if args.workload == "exhaustive":
        return run_exhaustive(args)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
