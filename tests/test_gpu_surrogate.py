"""GPU surrogate (hesp_surrogate_*) against the FP64 reference oracle/mlp_ref.py
on identical inputs (weights from the host-side initialiser, seeded levels and
makespans): initial weights bit-exact, forward outputs, loss and every
gradient within the tolerance of bf16 operands with FP32 accumulation
(relative error of each tensor <= 1e-2, cosine >= 0.999), one Adam step,
training that lowers the loss, and the selection / metric kernels against
numpy / scipy definitions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp_ref as R  # noqa: E402
from paper_1602_05510_b300 import hesp  # noqa: E402
from paper_1602_05510_b300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05510_b300 import build
    build.build()


def close(got, want, rel=1e-2, cos=0.999):
    got = np.asarray(got, np.float64).ravel()
    want = np.asarray(want, np.float64).ravel()
    nw = np.linalg.norm(want)
    assert np.linalg.norm(got - want) <= rel * max(nw, 1e-12), (np.linalg.norm(got - want), nw)
    if nw > 0 and np.linalg.norm(got) > 0:
        assert got @ want / (np.linalg.norm(got) * nw) >= cos


def batch(rng, B, T, NL):
    lv = rng.integers(0, NL, (B, T)).astype(np.int8)
    ms = np.exp(rng.normal(20.5, 0.3, B)).astype(np.int64)
    return lv, ms


SHAPES = [(10, 2, 64, 64), (816, 3, 512, 256), (120, 3, 128, 128), (40, 4, 128, 128), (33, 5, 64, 128), (20, 1, 64, 64)]


@pytest.mark.parametrize("T,NL,H,B", SHAPES)
def test_init_matches_host_initialiser(T, NL, H, B):
    s = hesp.Surrogate(T, NL, H, max_batch=max(B, 64), seed=17)
    ref = W.surrogate_init(17, T * NL, s.Fp, H)
    got = s.get(0)
    for k in s.PARTS:
        assert np.array_equal(got[k].reshape(-1), ref[k].reshape(-1)), k


@pytest.mark.parametrize("T,NL,H,B", SHAPES)
def test_forward_backward_parity(T, NL, H, B):
    rng = np.random.default_rng(T + H)
    s = hesp.Surrogate(T, NL, H, max_batch=B, seed=5)
    p = W.surrogate_init(5, T * NL, s.Fp, H)
    p["b1"] = (rng.standard_normal(H) * 0.05).astype(np.float32)
    p["b2"] = (rng.standard_normal(H) * 0.05).astype(np.float32)
    p["b3"] = np.array([0.1], np.float32)
    s.set(p)
    mu, sigma = 20.4, 0.25
    s.set_stats(mu, sigma)
    lv, ms = batch(rng, B, T, NL)
    pred = torch.empty(B, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    s.grad(torch.from_numpy(lv.reshape(-1).copy()).cuda(), torch.from_numpy(ms).cuda(), B, pred, loss)
    torch.cuda.synchronize()
    assert s.error_flag() == 0
    g = s.get(1)
    ref = R.MLPRef(p["W1"], p["b1"], p["W2"], p["b2"], p["w3"], float(p["b3"][0]))
    X = R.one_hot(lv, NL, s.Fp)
    t = (np.log(ms.astype(np.float64)) - mu) / sigma
    out = ref.backward(X, t)
    close(pred.cpu().numpy(), out["y"], rel=2e-3)
    assert abs(loss.item() - out["loss"]) <= 1e-2 * out["loss"]
    for k in s.PARTS:
        close(g[k], out["grads"][k])


def test_adam_step_parity():
    rng = np.random.default_rng(9)
    T, NL, H, B = 120, 3, 128, 128
    s = hesp.Surrogate(T, NL, H, max_batch=B, seed=2)
    p = W.surrogate_init(2, T * NL, s.Fp, H)
    s.set(p)
    s.set_stats(20.4, 0.25)
    lv, ms = batch(rng, B, T, NL)
    s.grad(torch.from_numpy(lv.reshape(-1).copy()).cuda(), torch.from_numpy(ms).cuda(), B)
    s.adam(1e-3)
    torch.cuda.synchronize()
    new = s.get(0)
    ref = R.MLPRef(p["W1"], p["b1"], p["W2"], p["b2"], p["w3"], float(p["b3"][0]))
    X = R.one_hot(lv, NL, s.Fp)
    g = ref.backward(X, (np.log(ms.astype(np.float64)) - 20.4) / 0.25)["grads"]
    for k in s.PARTS:
        want, _, _ = R.adam_step(np.asarray(p[k], np.float64), g[k].reshape(np.shape(p[k])), 0.0, 0.0, 1)
        d_got = np.asarray(new[k], np.float64) - p[k]
        d_want = want - p[k]
        # the first Adam step is lr * g / (|g| + eps): elements whose gradient is
        # near zero may differ, every other one moves by the same amount
        big = np.abs(g[k].reshape(np.shape(p[k]))) > 1e-4 * max(np.abs(g[k]).max(), 1e-30)
        assert np.mean(np.abs(d_got - d_want)[big] <= 1e-6) >= 0.99, k
        assert np.abs(d_got).max() <= 1.0001e-3


def test_training_lowers_loss_and_infer_is_consistent():
    rng = np.random.default_rng(1)
    T, NL, H = 120, 3, 256
    n = 8192
    lv = rng.integers(0, NL, (n, T)).astype(np.int8)
    # a target with structure: log makespan grows with the number of splits
    ms = np.exp(20.0 + 0.01 * lv.sum(1) + rng.normal(0, 0.01, n)).astype(np.int64)
    s = hesp.Surrogate(T, NL, H, max_batch=1024, seed=3)
    d_lv = torch.from_numpy(lv.reshape(-1).copy()).cuda()
    d_ms = torch.from_numpy(ms).cuda()
    s.fit_stats(d_ms)
    mu, sigma, _ = s.stats()
    assert abs(mu - np.log(ms).mean()) < 1e-9 and abs(sigma - np.log(ms).std()) < 1e-9
    losses = torch.empty(200, dtype=torch.float32, device="cuda")
    s.train(d_lv, d_ms, n, 1024, 200, lr=1e-3, seed=11, loss=losses)
    torch.cuda.synchronize()
    L = losses.cpu().numpy()
    assert s.error_flag() == 0
    assert L[-20:].mean() < 0.2 * L[:5].mean()
    pred = torch.empty(n, dtype=torch.float32, device="cuda")
    s.infer(d_lv, n, pred)
    torch.cuda.synchronize()
    t = (np.log(ms) - mu) / sigma
    assert np.corrcoef(pred.cpu().numpy(), t)[0, 1] > 0.9
    p = s.get(0)
    ref = R.MLPRef(p["W1"], p["b1"], p["W2"], p["b2"], p["w3"], float(p["b3"][0]))
    close(pred.cpu().numpy()[:512], ref.forward(R.one_hot(lv[:512], NL, s.Fp))["y"], rel=5e-3)


def test_select_topk_matches_definition():
    rng = np.random.default_rng(4)
    for n, k in ((1000, 10), (100000, 1000), (4 << 20, 40000)):
        keys = rng.standard_normal(n).astype(np.float32)
        keys[rng.choice(n, n // 10, replace=False)] = 0.25  # many ties
        d = torch.from_numpy(keys).cuda()
        idx = hesp.select_topk(d, k)
        torch.cuda.synchronize()
        want = np.sort(np.lexsort((np.arange(n), keys))[:k])
        assert np.array_equal(idx.cpu().numpy(), want)


def test_rank_metrics_match_scipy():
    import scipy.stats
    rng = np.random.default_rng(2)
    k = 5000
    pred = rng.standard_normal(k).astype(np.float32)
    pred[:100] = pred[100:200]  # ties
    ms = np.exp(20 + 0.3 * pred.astype(np.float64) + rng.normal(0, 0.2, k)).astype(np.int64)
    ms[300:320] = ms[320:340]
    mu, sigma = 20.0, 0.3
    rel, rho = hesp.rank_metrics(torch.from_numpy(pred).cuda(), torch.from_numpy(ms).cuda(), mu, sigma)
    want_rel = np.mean(np.abs(np.exp(pred.astype(np.float64) * sigma + mu) - ms) / ms)
    assert abs(rel - want_rel) <= 1e-9 * max(1.0, want_rel)
    assert abs(rho - scipy.stats.spearmanr(pred, ms).correlation) <= 1e-9


def test_make_cands_resimulates_selected_rows():
    lv = W.workload_levels("cfg1", 0, 512)
    d_lv = torch.from_numpy(lv.reshape(-1).copy()).cuda()
    keys = torch.from_numpy(np.random.default_rng(0).standard_normal(512).astype(np.float32)).cuda()
    idx = hesp.select_topk(keys, 40)
    cands = hesp.make_cands(idx, 8, 2048)
    plat = hesp.Platform(W.PLATFORMS["cfg1a"])
    ws = hesp.alloc_workspace(plat, 8, 2, 512)
    ms_sel, st_sel, _ = hesp.simulate_batch(plat, cands, d_lv, 40, 8, 2, ws)
    all_c = hesp.cands_tensor(8, 2048, np.arange(512) * 120)
    ms_all, st_all, _ = hesp.simulate_batch(plat, all_c, d_lv, 512, 8, 2, ws)
    torch.cuda.synchronize()
    assert (st_sel == 0).all() and (st_all == 0).all()
    assert torch.equal(ms_sel, ms_all[idx])


def test_checkpoint_roundtrip_and_resume(tmp_path):
    """hesp_surrogate_save / _load: the loaded handle holds the same
    parameters, Adam moments, step count and statistics, and training resumed
    from it is bit-identical to continuing the saved one; damaged files are
    refused."""
    rng = np.random.default_rng(12)
    T, NL, H, n = 120, 3, 128, 4096
    lv = rng.integers(0, NL, (n, T)).astype(np.int8)
    ms = np.exp(20.0 + 0.01 * lv.sum(1) + rng.normal(0, 0.01, n)).astype(np.int64)
    d_lv = torch.from_numpy(lv.reshape(-1).copy()).cuda()
    d_ms = torch.from_numpy(ms).cuda()
    a = hesp.Surrogate(T, NL, H, max_batch=512, seed=7)
    a.fit_stats(d_ms)
    a.train(d_lv, d_ms, n, 512, 25, lr=1e-3, seed=3)
    torch.cuda.synchronize()
    path = str(tmp_path / "sur.ckpt")
    a.save(path)
    b = hesp.Surrogate.load(path)
    assert (b.n_base, b.n_levels, b.H, b.max_batch) == (T, NL, H, 512)
    assert a.stats() == b.stats()
    for which in (0, 2, 3):
        ga, gb = a.get(which), b.get(which)
        for k in a.PARTS:
            assert np.array_equal(ga[k], gb[k]), (which, k)
    la = torch.empty(10, dtype=torch.float32, device="cuda")
    lb = torch.empty(10, dtype=torch.float32, device="cuda")
    a.train(d_lv, d_ms, n, 512, 10, lr=1e-3, seed=4, loss=la)
    b.train(d_lv, d_ms, n, 512, 10, lr=1e-3, seed=4, loss=lb)
    torch.cuda.synchronize()
    assert torch.equal(la, lb)
    pa, pb = a.get(0), b.get(0)
    assert all(np.array_equal(pa[k], pb[k]) for k in a.PARTS)
    raw = open(path, "rb").read()
    for bad in (raw[:-1], raw + b"x", raw[:100] + bytes([raw[100] ^ 1]) + raw[101:], b"NOTHESP!" + raw[8:]):
        p2 = str(tmp_path / "bad.ckpt")
        open(p2, "wb").write(bad)
        with pytest.raises(hesp.HespError):
            hesp.Surrogate.load(p2)


def _ref_forward_rows(ref, lv, NL, Fp, chunk=2048):
    """The FP64 reference forward over many rows, in row chunks (the dense
    one-hot matrix of every row at once would not fit): y, and per row the
    bound sum_h |w3_h| |A2_bh| used by the element-wise tolerance."""
    ys, bs = [], []
    for i in range(0, lv.shape[0], chunk):
        f = ref.forward(R.one_hot(lv[i:i + chunk], NL, Fp))
        ys.append(f["y"])
        bs.append(np.abs(f["A2"]) @ np.abs(ref.w3))
    return np.concatenate(ys), np.concatenate(bs)


# Inference chunks large enough that the persistent layer-1 and layer-2 GEMMs
# run several 128 x 256 tiles per CTA: 65,536 rows of the 816-task, 3-level
# input (1,024 tiles per layer) and 40,960 rows of the 5,984-task, 4-level
# input (23,936 features, 640 tiles).
@pytest.mark.parametrize("T,NL,M", [(816, 3, 65536), (5984, 4, 40960)])
def test_infer_elementwise_multi_tile(T, NL, M):
    rng = np.random.default_rng(T + M)
    H = 512
    s = hesp.Surrogate(T, NL, H, max_batch=M, seed=13)
    p = W.surrogate_init(13, T * NL, s.Fp, H)
    p["b1"] = (rng.standard_normal(H) * 0.1).astype(np.float32)
    p["b2"] = (rng.standard_normal(H) * 0.1).astype(np.float32)
    p["b3"] = np.array([0.05], np.float32)
    s.set(p)
    lv = rng.integers(0, NL, (M, T)).astype(np.int8)
    pred = torch.full((M,), float("nan"), dtype=torch.float32, device="cuda")
    s.infer(torch.from_numpy(lv.reshape(-1).copy()).cuda(), M, pred)
    torch.cuda.synchronize()
    assert s.error_flag() == 0
    ref = R.MLPRef(p["W1"], p["b1"], p["W2"], p["b2"], p["w3"], float(p["b3"][0]))
    y, bound = _ref_forward_rows(ref, lv, NL, s.Fp)
    got = pred.cpu().numpy().astype(np.float64)
    # per row: FP32 sums may move a bf16 rounding of A1 or A2 by one step
    # (2^-7 relative at most), so |dy| <= 2^-7 sum_h |w3_h| |A2_h|, plus the
    # FP32 error of the last dot product
    tol = 2.0 ** -7 * bound + 1e-5 * np.maximum(1.0, np.abs(y))
    assert np.all(np.abs(got - y) <= tol), float(np.max(np.abs(got - y) / tol))


def test_grad_elementwise_multi_tile_5984_tasks():
    """Forward and backward of the 5,984-task, 4-level surrogate on a batch
    of 512: the weight gradient dW1 = dZ1^T X is a 512 x 23,936 GEMM of 376
    output tiles.  Biases keep every ReLU clearly active (checked below), so
    the masks agree with the reference and each bf16-rounded backward
    activation dZ1 is within one bf16 step (2^-7 relative) of the
    reference's; every element of dW1 must then lie within
    2^-6 sum_b |dZ1_bh| X_bf of the FP64 value."""
    rng = np.random.default_rng(4)
    T, NL, H, B = 5984, 4, 512, 512
    s = hesp.Surrogate(T, NL, H, max_batch=B, seed=21)
    p = W.surrogate_init(21, T * NL, s.Fp, H)
    p["b1"] = np.full(H, 6.0, np.float32)
    p["b2"] = np.full(H, 60.0, np.float32)
    p["b3"] = np.array([0.1], np.float32)
    s.set(p)
    s.set_stats(20.4, 0.25)
    lv, ms = batch(rng, B, T, NL)
    pred = torch.empty(B, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    s.grad(torch.from_numpy(lv.reshape(-1).copy()).cuda(), torch.from_numpy(ms).cuda(), B, pred, loss)
    torch.cuda.synchronize()
    assert s.error_flag() == 0
    g = s.get(1)
    ref = R.MLPRef(p["W1"], p["b1"], p["W2"], p["b2"], p["w3"], float(p["b3"][0]))
    X = R.one_hot(lv, NL, s.Fp)
    f = ref.forward(X)
    # precondition of the element-wise bound: no pre-activation near the ReLU cut
    pre1 = X @ f["W1r"].T + ref.b1
    pre2 = f["A1"] @ f["W2r"].T + ref.b2
    assert pre1.min() > 1.0 and pre2.min() > 1.0
    t = (np.log(ms.astype(np.float64)) - 20.4) / 0.25
    out = ref.backward(X, t)
    y_gpu = pred.cpu().numpy().astype(np.float64)
    close(y_gpu, out["y"], rel=2e-3)
    assert abs(loss.item() - out["loss"]) <= 1e-2 * out["loss"]
    for k in s.PARTS:
        close(g[k], out["grads"][k])
    # The backward pass starts from dy = 2 (y - t) / B; a bf16 step of A2
    # moves the GPU's y slightly, which would move roundings of dZ2.  Shifting
    # the targets by y_ref - y_gpu gives the reference the GPU's dy, so dZ2
    # and dZ1 differ from the GPU's by FP32-vs-FP64 rounding alone.
    out = ref.backward(X, t + out["y"] - y_gpu)
    bound = np.abs(out["dZ1"]).T @ X
    got = np.asarray(g["W1"], np.float64)
    want = out["grads"]["W1"]
    assert np.all(np.abs(got - want) <= 2.0 ** -6 * bound + 1e-12), float(np.max(np.abs(got - want) - 2.0 ** -6 * bound))
