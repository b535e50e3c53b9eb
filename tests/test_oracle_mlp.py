"""Pins of the FP64 surrogate reference (oracle/mlp_ref.py), CPU only:
bf16 rounding against torch's conversion, a hand-derived one-sample network,
finite differences of every gradient, Adam's closed-form first step, one-hot
encoding, and the initialiser's range."""
import numpy as np
import pytest
import torch

from oracle import mlp_ref as R
from paper_1602_05510_b300 import workloads as W


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10 ** rng.uniform(-8, 8, 20000),
                        [0.0, -0.0, 1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 65504.0, 3.0e38]])
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(R.bf16_round(x), want)


def test_one_hot():
    lv = np.array([[0, 2, 1], [1, 1, 0]])
    X = R.one_hot(lv, 3, 12)
    assert X.shape == (2, 12) and (X.sum(1) == 3).all()
    assert X[0, 0] == X[0, 5] == X[0, 7] == 1 and X[0, 9:].sum() == 0
    assert X[1, 1] == X[1, 4] == X[1, 6] == 1


def _hand():
    return R.MLPRef(W1=[[0.5, 2.0]], b1=[0.25], W2=[[-1.5]], b2=[4.0], w3=[3.0], b3=0.5)


@pytest.mark.parametrize("rnd", [True, False])
def test_hand_derived_one_sample(rnd):
    # x = one_hot(level 1 of 2): z1 = 2 + .25, a2 = -1.5 * 2.25 + 4 = .625,
    # y = 3 * .625 + .5 = 2.375; t = 1: L = 1.375^2, dy = 2.75, dz2 = 8.25,
    # dW2 = 8.25 * 2.25, dz1 = 8.25 * -1.5, dW1 = [0, dz1]
    m = _hand()
    X = R.one_hot(np.array([[1]]), 2)
    out = m.backward(X, np.array([1.0]), round_bf16=rnd)
    g = out["grads"]
    assert out["y"][0] == 2.375 and out["loss"] == 1.890625
    assert g["w3"][0] == 1.71875 and g["b3"][0] == 2.75
    assert g["W2"][0, 0] == 18.5625 and g["b2"][0] == 8.25
    assert g["W1"].tolist() == [[0.0, -12.375]] and g["b1"][0] == -12.375


def test_relu_cut_stops_gradient():
    m = R.MLPRef(W1=[[0.5, 2.0]], b1=[0.25], W2=[[-3.0]], b2=[1.0], w3=[3.0], b3=0.5)
    out = m.backward(R.one_hot(np.array([[1]]), 2), np.array([1.0]))
    assert out["y"][0] == 0.5
    assert not out["grads"]["W1"].any() and not out["grads"]["W2"].any() and not out["grads"]["w3"].any()
    assert out["grads"]["b3"][0] == 2 * (0.5 - 1.0)


def test_finite_differences():
    rng = np.random.default_rng(4)
    T, NL, H, B = 5, 3, 7, 9
    F = T * NL
    m = R.MLPRef(W1=rng.standard_normal((H, F + 1)) * 0.5, b1=rng.standard_normal(H) * 0.1,
                 W2=rng.standard_normal((H, H)) * 0.5, b2=rng.standard_normal(H) * 0.1,
                 w3=rng.standard_normal(H), b3=0.3)
    X = R.one_hot(rng.integers(0, NL, (B, T)), NL, F + 1)
    t = rng.standard_normal(B)
    g = m.backward(X, t, round_bf16=False)["grads"]
    h = 1e-6
    for name, P in m.params().items():
        flat = P.reshape(-1)
        for idx in rng.choice(flat.size, min(flat.size, 12), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            if name == "b3":
                m.b3 = flat[idx]
            lp = m.loss(X, t, round_bf16=False)
            flat[idx] = old - h
            if name == "b3":
                m.b3 = flat[idx]
            lm = m.loss(X, t, round_bf16=False)
            flat[idx] = old
            if name == "b3":
                m.b3 = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name].reshape(-1)[idx]) <= 1e-6 * (1 + abs(fd)), (name, idx)


def test_adam_first_step_closed_form():
    # k = 1: m_hat = g, v_hat = g^2, so p1 = p0 - lr g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p, m, v = R.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1)
    assert np.allclose(p, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_he_uniform_init():
    w = W.he_uniform(3, 0, 64, 130, 120, 120)
    b = np.sqrt(6 / 120)
    assert w.dtype == np.float32 and abs(w[:, :120]).max() <= b and (w[:, 120:] == 0).all()
    assert abs(w[:, :120].mean()) < 0.02 and abs(w[:, :120].std() - b / np.sqrt(3)) < 0.01
    p = W.surrogate_init(3, 2448, 2496, 512)
    assert p["W1"].shape == (512, 2496) and p["W2"].shape == (512, 512) and p["w3"].shape == (512,)
