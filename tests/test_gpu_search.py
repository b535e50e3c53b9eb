"""Search drivers on the GPU (small budgets): plain random search and
surrogate-guided search both return monotone best-so-far traces whose best
makespans are real simulation results, and the surrogate rounds report
finite relative error and rank correlation."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1602_05510_b300 import hesp  # noqa: E402
from paper_1602_05510_b300 import search as S  # noqa: E402
from paper_1602_05510_b300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05510_b300 import build
    build.build()


def test_random_and_surrogate_search_small():
    spec = W.PLATFORMS["cfg1a"]
    r = S.random_search(spec, 8, 2048, 3, seed=5, budget_s=0.0, per_launch=2048)  # one launch
    cfg = S.SurrogateConfig(hidden=128, batch=1024, warmup_launches=2, warmup_steps=50, steps_per_round=10,
                            proposals=16384, elites=16, label_cap=1 << 16)
    s = S.surrogate_search(spec, 8, 2048, 3, seed=5, budget_s=3.0, per_launch=2048, cfg=cfg)
    assert len(r.best) == 1 and len(s.best) >= 3
    for log in (r, s):
        assert all(a >= b for a, b in zip(log.best, log.best[1:]))
        assert all(a <= b for a, b in zip(log.events, log.events[1:]))
    assert s.metrics and all(np.isfinite(m["rel_err"]) and -1 <= m["spearman"] <= 1 for m in s.metrics)
    # the random arm's best is the makespan of one of its uniform candidates
    lv = W.uniform_levels(5, 0, 2048, 120, 3)
    pl = O.make_platform(spec)
    first = min(O.simulate(pl, 8, 2048, lv[c], schedule=False)["makespan"] for c in range(0, 2048, 97))
    assert r.best[0] <= first


def test_trained_surrogate_gains_over_unranked_proposals():
    """What the learned part adds: after training on simulator labels, the
    proposals the surrogate ranks best simulate to clearly shorter makespans
    than the same number of proposals taken without it (the method's plain
    random sampling), and the exact makespans of a held-out set correlate
    with the predictions."""
    from paper_1602_05510_b300 import hesp

    spec = W.PLATFORMS["cfg1a"]
    n, b, NL, nb = 8, 2048, 3, 120
    n_lab, n_prop, k = 16384, 16384, 512
    sim = S.Simulator(spec, n, b, NL - 1, n_lab)
    lab = torch.empty(n_lab * nb, dtype=torch.int8, device="cuda")
    hesp.generate_candidates(hesp.GEN_UNIFORM, 21, 0, n_lab, n, b, NL, lab)
    ms, st, _ = sim.run(lab)
    assert bool((st == 0).all())
    lab_ms = ms.clone()
    sur = hesp.Surrogate(nb, NL, 256, 2048, seed=3)
    sur.fit_stats(lab_ms)
    mu, sigma, _ = sur.stats()
    sur.train(lab, lab_ms, n_lab, 2048, 400, 1e-3, seed=4)
    prop = torch.empty(n_prop * nb, dtype=torch.int8, device="cuda")
    hesp.generate_candidates(hesp.GEN_UNIFORM, 22, 0, n_prop, n, b, NL, prop)
    pred = torch.empty(n_prop, dtype=torch.float32, device="cuda")
    sur.infer(prop, n_prop, pred)
    ms_all, st_all, _ = sim.run(prop)  # held-out exact makespans of every proposal
    torch.cuda.synchronize()
    assert bool((st_all == 0).all()) and sur.error_flag() == 0
    idx = hesp.select_topk(pred, k)
    top = ms_all[idx].double()
    plain = ms_all[:k].double()  # proposals are independent draws: the first k are a random sample
    assert top.mean() < plain.mean() - 3 * plain.std() / np.sqrt(k)
    assert top.min() <= plain.min()
    rel, rho = hesp.rank_metrics(pred, ms_all, mu, sigma)
    assert rho > 0.5 and rel < 0.05


def test_best_candidate_matches_definition():
    """hesp_best_candidate: the least makespan among successful candidates
    and the lowest index holding it (offset by the batch's first global
    index), with ties, failed candidates and an all-failed batch."""
    rng = np.random.default_rng(8)
    for n, first in ((1, 0), (1000, 7), (70000, 123456789)):
        ms = rng.integers(10 ** 9, 10 ** 9 + 50, n).astype(np.int64)  # many ties
        st = np.where(rng.random(n) < 0.2, -1, 0).astype(np.int32)
        st[0] = 0
        out = hesp.best_candidate(torch.from_numpy(ms).cuda(), torch.from_numpy(st).cuda(), first).cpu().numpy()
        ok = st == 0
        m = int(ms[ok].min())
        assert out.tolist() == [m, first + int(np.flatnonzero(ok & (ms == m))[0])]
    st = np.full(16, -1, np.int32)
    out = hesp.best_candidate(torch.zeros(16, dtype=torch.int64, device="cuda"), torch.from_numpy(st).cuda(), 5)
    assert out.cpu().tolist() == [np.iinfo(np.int64).max, -1]


def test_solver_seeded_surrogate_search_small():
    """The surrogate arm started from the iterative solver's descent: its
    first records follow the solver from the unsplit partition (so its best
    is at most the unsplit makespan), later rounds report the error and
    rank correlation on a held-out uniform sample, and the best is a real
    simulation result (the oracle agrees on the unsplit partition)."""
    spec = W.PLATFORMS["cfg1a"]
    cfg = S.SurrogateConfig(hidden=128, batch=1024, warmup_steps=50, steps_per_round=10, proposals=8192,
                            elites=16, label_cap=1 << 16, p_mut=0.01, start="solver", heldout=256)
    s = S.surrogate_search(spec, 8, 2048, 3, seed=5, budget_s=4.0, per_launch=1024, cfg=cfg)
    unsplit = O.simulate(O.make_platform(spec), 8, 2048, np.zeros(120, np.int8), schedule=False)["makespan"]
    assert s.best[0] <= unsplit
    assert all(a >= b for a, b in zip(s.best, s.best[1:]))
    assert s.metrics
    for m in s.metrics:
        assert np.isfinite(m["heldout_rel_err"]) and -1 <= m["heldout_spearman"] <= 1
