"""Partition search on the GPU: plain batched random search, and
surrogate-guided search (the partition stage of HeSP's iterative solver,
Sec. 2.1, with proposals ranked by the learned surrogate and only the
best-ranked slice simulated exactly).

Orchestration only: every step runs in libhesp.so kernels (candidate and
mutant generation, simulation, surrogate training and inference, top-k
selection, gathers, rank metrics).  The host keeps the bookkeeping that
needs a few bytes per candidate: the best makespan found and the elite set.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import hesp
from . import workloads as W


@dataclass
class SearchLog:
    arm: str
    times: List[float] = field(default_factory=list)    # seconds since start
    best: List[int] = field(default_factory=list)       # best makespan so far (ns)
    events: List[int] = field(default_factory=list)     # task-events simulated so far
    simulated: List[int] = field(default_factory=list)  # candidates simulated so far
    metrics: List[dict] = field(default_factory=list)   # per-round surrogate metrics

    def best_at(self, t: float) -> Optional[int]:
        b = None
        for tt, v in zip(self.times, self.best):
            if tt <= t:
                b = v
        return b

    def time_to_reach(self, target: int) -> Optional[float]:
        for tt, v in zip(self.times, self.best):
            if v <= target:
                return tt
        return None


class Simulator:
    """Batched exact simulation of fixed-size candidates of one workload."""

    def __init__(self, spec, n_tiles, b, max_level, per_launch, task_cap=0, ws_bytes=None):
        import torch
        self.plat = hesp.Platform(spec)
        self.n_tiles, self.b, self.max_level, self.per_launch, self.task_cap = n_tiles, b, max_level, per_launch, task_cap
        self.nb = W.base_count(n_tiles)
        self.ws = hesp.alloc_workspace(self.plat, n_tiles, max_level, per_launch, task_cap, max_bytes=ws_bytes)
        self.cands = hesp.cands_tensor(n_tiles, b, np.arange(per_launch, dtype=np.int64) * self.nb)
        self.ms = torch.empty(per_launch, dtype=torch.int64, device="cuda")
        self.st = torch.empty(per_launch, dtype=torch.int32, device="cuda")
        self.nt = torch.empty(per_launch, dtype=torch.int64, device="cuda")

    def run(self, levels, n=None, cands=None):
        n = self.per_launch if n is None else n
        hesp.simulate_batch(self.plat, self.cands if cands is None else cands, levels, n, self.n_tiles,
                            self.max_level, self.ws, makespan=self.ms, status=self.st, ntasks=self.nt,
                            task_cap=self.task_cap)
        return self.ms[:n], self.st[:n], self.nt[:n]


def random_search(spec, n_tiles, b, n_levels, seed, budget_s, per_launch=4096, task_cap=0, ws_bytes=None,
                  sim: Optional[Simulator] = None) -> SearchLog:
    """Uniform random partition vectors, per_launch per simulation launch,
    until budget_s of wall time have passed."""
    import torch
    sim = sim or Simulator(spec, n_tiles, b, n_levels - 1, per_launch, task_cap, ws_bytes)
    nb = sim.nb
    levels = torch.empty(per_launch * nb, dtype=torch.int8, device="cuda")
    log = SearchLog("random")
    best, events, done, k = None, 0, 0, 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while True:
        hesp.generate_candidates(hesp.GEN_UNIFORM, seed, k * per_launch, per_launch, n_tiles, b, n_levels, levels)
        ms, st, nt = sim.run(levels)
        m, ev = (int(v) for v in hesp.best_makespan(ms, st, nt).cpu().numpy())
        events += ev
        done += per_launch
        best = m if best is None else min(best, m)
        el = time.perf_counter() - t0
        log.times.append(el)
        log.best.append(best)
        log.events.append(events)
        log.simulated.append(done)
        k += 1
        if el >= budget_s:
            break
    return log


@dataclass
class SurrogateConfig:
    hidden: int = 512
    batch: int = 4096
    lr: float = 1e-3
    warmup_launches: int = 2       # random launches labelled before the first training
    warmup_steps: int = 300
    steps_per_round: int = 60
    proposals: int = 131072        # proposals ranked per round
    random_fraction: float = 0.25  # share of proposals drawn uniformly (the rest mutate elites)
    elites: int = 64
    p_mut: float = 0.01
    label_cap: int = 1 << 20
    infer_chunk: int = 16384       # rows per inference launch (activation buffers)
    use_surrogate: bool = True     # False: simulate random mutants (the same search without the model)
    # "random": the first labels come from warmup_launches uniform launches;
    # "solver": from the paper's iterative solver (CP selection, Hard
    # sampling) run from the unsplit partition to its first local optimum --
    # every partition it simulates is a label, and its elites seed the rounds
    start: str = "random"
    solver_iters: int = 1000       # cap on the solver's iterations in "solver" mode
    heldout: int = 0               # uniform partitions simulated once, never trained on: each round's
                                   # relative error and Spearman rank correlation on them


def surrogate_search(spec, n_tiles, b, n_levels, seed, budget_s, per_launch=4096, cfg: SurrogateConfig = None,
                     task_cap=0, ws_bytes=None, sim: Optional[Simulator] = None) -> SearchLog:
    """Each round: mutate the elite partitions (and draw some uniform ones),
    rank all proposals with the surrogate, simulate the per_launch best-ranked
    exactly, add them to the labels, retrain briefly."""
    import torch
    cfg = cfg or SurrogateConfig()
    nb = W.base_count(n_tiles)
    P = cfg.proposals
    n_rand = int(P * cfg.random_fraction) // 64 * 64
    lab_lv = torch.empty(cfg.label_cap * nb, dtype=torch.int8, device="cuda")
    lab_ms = torch.empty(cfg.label_cap, dtype=torch.int64, device="cuda")
    host_ms = np.empty(cfg.label_cap, np.int64)
    prop = torch.empty(P * nb, dtype=torch.int8, device="cuda")
    pred = torch.empty(P, dtype=torch.float32, device="cuda")
    parents = torch.empty(cfg.elites * nb, dtype=torch.int8, device="cuda")
    sur = hesp.Surrogate(nb, n_levels, cfg.hidden, max(cfg.batch, cfg.infer_chunk), seed=seed)
    log = SearchLog("surrogate" if cfg.use_surrogate else "mutation")
    n_lab, best, events, done, rnd = 0, None, 0, 0, 0
    big = np.iinfo(np.int64).max

    def add(levels_rows, ms, st, nt, count):
        # failed candidates (none are expected) keep the largest makespan
        nonlocal n_lab, best, events, done
        take = min(count, cfg.label_cap - n_lab)
        if take > 0:
            lab_lv[n_lab * nb:(n_lab + take) * nb].copy_(levels_rows[:take * nb])
            lab_ms[n_lab:n_lab + take].copy_(ms[:take])
            h_ms, h_st = ms[:take].cpu().numpy(), st[:take].cpu().numpy()
            host_ms[n_lab:n_lab + take] = np.where(h_st == 0, h_ms, big)
            n_lab += take
        m, ev = (int(v) for v in hesp.best_makespan(ms, st, nt).cpu().numpy())
        events += ev
        done += count
        if m != big:
            best = m if best is None else min(best, m)

    def record(t0, extra=None):
        log.times.append(time.perf_counter() - t0)
        log.best.append(best)
        log.events.append(events)
        log.simulated.append(done)
        if extra is not None:
            log.metrics.append(extra)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if cfg.start == "solver":
        # the solver's descent from the unsplit partition: each iteration's
        # current partition and every moved partition it simulated are labels
        sv = IterativeSolver(spec, n_tiles, b, n_levels, hesp.SOLVER_CP, hesp.PICK_HARD, task_cap, ws_bytes)
        sv.start(levels=np.zeros(nb, np.int8))
        for it in range(cfg.solver_iters):
            if time.perf_counter() - t0 >= budget_s:
                break
            chosen, k, _, _ = sv.iterate(seed, it)
            add(sv.cur_before, sv.cur_ms, sv.cur_st, None, 1)
            if k:
                add(sv.rows, sv.ms[:k], sv.st[:k], sv.nt[:k], k)
            record(t0)
            if chosen is None:
                break
        del sv
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    sim = sim or Simulator(spec, n_tiles, b, n_levels - 1, per_launch, task_cap, ws_bytes)
    if cfg.start != "solver":
        # warm-up labels from uniform random partitions
        for w in range(cfg.warmup_launches):
            hesp.generate_candidates(hesp.GEN_UNIFORM, seed, w * per_launch, per_launch, n_tiles, b, n_levels,
                                     prop)
            ms, st, nt = sim.run(prop)
            add(prop, ms, st, nt, per_launch)
            record(t0)
    ho = None
    if cfg.heldout > 0:
        # a held-out uniform sample (its own SplitMix64 stream), simulated once
        H_ = cfg.heldout
        ho_lv = torch.empty(H_ * nb, dtype=torch.int8, device="cuda")
        ho_ms = torch.empty(H_, dtype=torch.int64, device="cuda")
        ho_st = torch.empty(H_, dtype=torch.int32, device="cuda")
        hesp.generate_candidates(hesp.GEN_UNIFORM, seed + 11, 0, H_, n_tiles, b, n_levels, ho_lv)
        for i in range(0, H_, per_launch):
            c = min(per_launch, H_ - i)
            ms, st, _ = sim.run(ho_lv[i * nb:], c)
            ho_ms[i:i + c].copy_(ms)
            ho_st[i:i + c].copy_(st)
        ho_ok = ho_st == 0
        ho = (ho_lv, ho_ms, ho_ok, torch.empty(H_, dtype=torch.float32, device="cuda"))
    sur.fit_stats(lab_ms[:n_lab])
    mu, sigma, _ = sur.stats()
    if cfg.use_surrogate:
        sur.train(lab_lv, lab_ms, n_lab, cfg.batch, cfg.warmup_steps, cfg.lr, seed=seed + 1)
    first_prop = 1 << 40
    while time.perf_counter() - t0 < budget_s:
        # proposals: mutants of the elites, plus some uniform draws
        el_idx = np.argsort(host_ms[:n_lab], kind="stable")[:cfg.elites]
        hesp.gather_rows(lab_lv, torch.from_numpy(el_idx.astype(np.int64)).cuda(), nb, parents)
        n_mut = P - n_rand
        hesp.generate_mutants(parents, len(el_idx), nb, n_levels, cfg.p_mut, seed + 7, first_prop + rnd * P, n_mut,
                              prop)
        if n_rand:
            hesp.generate_candidates(hesp.GEN_UNIFORM, seed + 3, rnd * n_rand, n_rand, n_tiles, b, n_levels,
                                     prop[n_mut * nb:])
        if cfg.use_surrogate:
            sur.infer(prop, P, pred)
            idx = hesp.select_topk(pred, per_launch)
        else:
            # the same proposals, a random sample of them simulated (proposals
            # are independent draws, so the first ones of each kind are one)
            k_rand = int(per_launch * cfg.random_fraction) if n_rand else 0
            idx = torch.from_numpy(np.concatenate([np.arange(per_launch - k_rand),
                                                   n_mut + np.arange(k_rand)]).astype(np.int64)).cuda()
        cands = hesp.make_cands(idx, n_tiles, b)
        ms, st, nt = sim.run(prop, per_launch, cands)
        rel = rho = float("nan")
        if cfg.use_surrogate:
            sel_pred = hesp.gather_f32(pred, idx)
            okm = st == 0
            if int(okm.sum().item()) > 1:
                rel, rho = hesp.rank_metrics(sel_pred[okm], ms[okm], mu, sigma)
        rows = hesp.gather_rows(prop, idx, nb)
        add(rows, ms, st, nt, per_launch)
        m = {"round": rnd, "rel_err": rel, "spearman": rho, "labels": n_lab}
        if cfg.use_surrogate and ho is not None:
            ho_lv, ho_ms, ho_ok, ho_pred = ho
            sur.infer(ho_lv, cfg.heldout, ho_pred)
            m["heldout_rel_err"], m["heldout_spearman"] = hesp.rank_metrics(ho_pred[ho_ok], ho_ms[ho_ok], mu, sigma)
        record(t0, m)
        if cfg.use_surrogate:
            sur.train(lab_lv, lab_ms, n_lab, cfg.batch, cfg.steps_per_round, cfg.lr, seed=seed + 100 + rnd)
        rnd += 1
    return log


@dataclass
class SolverStep:
    levels: np.ndarray        # partition at the start of the iteration
    makespan: int
    moves: List[int]          # candidate move codes (2 t + d)
    makespans: List[int]      # simulated makespan of each moved partition
    chosen: Optional[int]     # applied move code, None at a local optimum


class IterativeSolver:
    """HeSP's iterative partition solver (Sec. 2.1 "Iterative solver") on one
    GPU.  Each iteration: the schedule stage simulates the current partition
    (with critical-path flags), the partition stage lists the candidate moves
    (selection All / CP / Shallow), simulates every moved partition in one
    batched launch, and applies the best (Hard) or a score-proportional draw
    (Soft).  Per iteration the host reads back two numbers (the move count
    and the chosen move).

    factors=True: the partition is one factor k in 1 .. n_levels per base
    task (one-level k-way partitions, p = 1/k, hesp_simulate_factors); a move
    makes a task's p finer (k + 1) or coarser (k - 1, merging it back at
    k = 1)."""

    def __init__(self, spec, n_tiles, b, n_levels, mode, pick, task_cap=0, ws_bytes=None, order=0, select=0,
                 rp_seed=0, factors=False):
        import torch
        self.plat = hesp.Platform(spec, order=order, select=select, rp_seed=rp_seed)
        self.n, self.b, self.NL, self.mode, self.pick, self.task_cap = n_tiles, b, n_levels, mode, pick, task_cap
        self.factors = factors
        self.lo, self.hi = (1, n_levels) if factors else (0, n_levels - 1)
        nb = self.nb = W.base_count(n_tiles)
        self.max_moves = 2 * nb
        if factors:
            self.ws = hesp.alloc_workspace_factors(self.plat, n_tiles, n_levels, self.max_moves, task_cap)
        else:
            self.ws = hesp.alloc_workspace(self.plat, n_tiles, n_levels - 1, self.max_moves, task_cap,
                                           max_bytes=ws_bytes)
        dev = "cuda"
        self.cur = torch.zeros(nb, dtype=torch.int8, device=dev)
        self.rows = torch.empty(self.max_moves * nb, dtype=torch.int8, device=dev)
        self.moves = torch.empty(self.max_moves, dtype=torch.int32, device=dev)
        self.count = torch.zeros(1, dtype=torch.int64, device=dev)
        self.crit = torch.zeros(nb, dtype=torch.int8, device=dev)
        self.cur_ms = torch.empty(1, dtype=torch.int64, device=dev)
        self.cur_st = torch.empty(1, dtype=torch.int32, device=dev)
        self.ms = torch.empty(self.max_moves, dtype=torch.int64, device=dev)
        self.st = torch.empty(self.max_moves, dtype=torch.int32, device=dev)
        self.nt = torch.empty(self.max_moves, dtype=torch.int64, device=dev)
        self.chosen = torch.empty(1, dtype=torch.int64, device=dev)
        self.cur_before = torch.empty(nb, dtype=torch.int8, device=dev)  # the last iteration's start
        self.cands_rows = hesp.cands_tensor(n_tiles, b, np.arange(self.max_moves, dtype=np.int64) * nb)
        self.cand_cur = hesp.cands_tensor(n_tiles, b, np.zeros(1, np.int64))

    def start(self, levels=None, seed=0, draw=0):
        """Set the current partition: `levels` (host), or the uniform draw
        `draw` of the SplitMix64 stream `seed`."""
        import torch
        if levels is not None:
            self.cur.copy_(torch.from_numpy(np.ascontiguousarray(levels, np.int8)))
        elif self.factors:
            self.cur.copy_(torch.from_numpy(W.uniform_factors(seed, draw, 1, self.nb, self.NL)[0]))
        else:
            hesp.generate_candidates(hesp.GEN_UNIFORM, seed, draw, 1, self.n, self.b, self.NL, self.cur)

    def schedule_stage(self):
        if self.factors:
            hesp.simulate_factors(self.plat, self.cand_cur, self.cur, 1, self.n, self.NL, self.b, self.ws,
                                  makespan=self.cur_ms, status=self.cur_st, task_cap=self.task_cap, crit=self.crit)
        else:
            hesp.simulate_critical(self.plat, self.cand_cur, self.cur, 1, self.n, self.NL - 1, self.ws, self.crit,
                                   makespan=self.cur_ms, status=self.cur_st, task_cap=self.task_cap)

    def simulate_rows(self, k):
        if self.factors:
            hesp.simulate_factors(self.plat, self.cands_rows, self.rows, k, self.n, self.NL, self.b, self.ws,
                                  makespan=self.ms, status=self.st, ntasks=self.nt, task_cap=self.task_cap)
        else:
            hesp.simulate_batch(self.plat, self.cands_rows, self.rows, k, self.n, self.NL - 1, self.ws,
                                makespan=self.ms, status=self.st, ntasks=self.nt, task_cap=self.task_cap)

    def iterate(self, seed, iteration, trace=False):
        """One iteration from the current partition.  Returns (chosen move or
        None, moves simulated, task-events simulated, SolverStep if trace)."""
        import torch
        if trace:
            lv0 = self.cur.cpu().numpy().copy()
        self.cur_before.copy_(self.cur)
        self.schedule_stage()
        hesp.solver_moves_range(self.cur, self.nb, self.lo, self.hi, self.mode, self.crit, self.moves, self.count,
                                self.rows)
        k = int(self.count.item())
        step = None
        if trace:
            m0 = int(self.cur_ms.item())
        if k == 0:
            if trace:
                step = SolverStep(lv0, m0, [], [], None)
            return None, 0, 0, step
        self.simulate_rows(k)
        if trace:
            mv = self.moves[:k].cpu().numpy().tolist()
            mss = self.ms[:k].cpu().numpy().tolist()
        hesp.solver_pick(self.ms, self.st, self.moves, self.count, self.pick, seed, iteration, self.cur_ms, self.cur,
                         self.chosen)
        _, ev = hesp.best_makespan(self.ms[:k], self.st[:k], self.nt[:k])
        vals = torch.stack([self.chosen[0], ev]).cpu().numpy()
        ch = int(vals[0])
        if ch == -2:
            raise hesp.HespError(-6, "hesp_solver_pick (score sum >= 2^64)")
        chosen = None if ch < 0 else ch
        if trace:
            step = SolverStep(lv0, m0, mv, mss, chosen)
        return chosen, k, int(vals[1]), step

    def solve(self, levels0, seed, iterations):
        """Up to `iterations` iterations from levels0; the trace of each."""
        self.start(levels0)
        steps = []
        for it in range(iterations):
            chosen, _, _, step = self.iterate(seed, it, trace=True)
            steps.append(step)
            if chosen is None:
                break
        return steps


def iterative_search(spec, n_tiles, b, n_levels, mode, pick, seed, budget_s, task_cap=0, ws_bytes=None,
                     solver: Optional[IterativeSolver] = None, first=None) -> SearchLog:
    """The iterative solver as a search arm: from a start partition, iterate
    to a local optimum, then restart, until budget_s of wall time have
    passed.  Restart 0 starts from `first` (host levels) when given, every
    other restart r from draw r of the uniform SplitMix64 stream `seed`.
    Soft draws use (seed + r, iteration)."""
    import torch
    sv = solver or IterativeSolver(spec, n_tiles, b, n_levels, mode, pick, task_cap, ws_bytes)
    names = {hesp.SOLVER_ALL: "all", hesp.SOLVER_CP: "cp", hesp.SOLVER_SHALLOW: "shallow"}
    log = SearchLog("iterative-%s-%s" % (names[mode], "hard" if pick == hesp.PICK_HARD else "soft"))
    best, events, done, r = None, 0, 0, 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        if r == 0 and first is not None:
            sv.start(levels=first)
        else:
            sv.start(seed=seed, draw=r)
        it = 0
        while time.perf_counter() - t0 < budget_s:
            chosen, k, ev, _ = sv.iterate(seed + r, it)
            events += ev
            done += k
            m = int(sv.cur_ms.item())
            best = m if best is None else min(best, m)
            log.times.append(time.perf_counter() - t0)
            log.best.append(best)
            log.events.append(events)
            log.simulated.append(done)
            it += 1
            if chosen is None:
                break
        log.metrics.append({"restart": r, "iterations": it, "makespan": int(sv.cur_ms.item())})
        r += 1
    return log
