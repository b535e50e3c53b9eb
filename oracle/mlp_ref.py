"""FP64 reference of the learned surrogate: a small MLP that maps a partition
vector (one split level per base task, one-hot encoded) to a predicted
standardised log-makespan, trained with MSE and Adam.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The surrogate is not
part of the paper; it ranks the partition proposals that HeSP's search (Sec. 2.1
"Iterative solver", partition stage) would otherwise have to simulate one by one.

Definition (the CUDA kernels implement the same one):
  X   = one_hot(levels)                  [B, F], F = T_base * n_levels (padded
                                          with zero columns to Fp)
  A1  = bf16(relu(X bf16(W1)^T + b1))     [B, H]
  A2  = bf16(relu(A1 bf16(W2)^T + b2))    [B, H]
  y   = A2 w3 + b3                        [B]
  L   = mean_b (y_b - t_b)^2
Backward (bf16 operands where the GPU feeds tensor cores, FP32/FP64 sums):
  dy  = 2 (y - t) / B
  dw3 = A2^T dy, db3 = sum dy
  dZ2 = bf16(dy w3^T * [A2 > 0]);   dW2 = dZ2^T A1;  db2 = sum_b dZ2
  dZ1 = bf16((dZ2 bf16(W2)) * [A1 > 0]); dW1 = dZ1^T X; db1 = sum_b dZ1
Adam (FP32 masters): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
  p -= lr * (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps).
Here every sum is evaluated in float64 on the same bf16-rounded operands; with
round_bf16=False all rounding is skipped (used by the finite-difference pins).
"""
from __future__ import annotations

import numpy as np


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64.
    Values are first taken to float32, as on the GPU."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    nan = np.isnan(f)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def one_hot(levels: np.ndarray, n_levels: int, f_pad: int | None = None) -> np.ndarray:
    lv = np.asarray(levels, dtype=np.int64)
    B, T = lv.shape
    F = T * n_levels
    X = np.zeros((B, f_pad or F), dtype=np.float64)
    cols = np.arange(T)[None, :] * n_levels + lv
    X[np.arange(B)[:, None], cols] = 1.0
    return X


class MLPRef:
    """Parameters are float64 copies of the FP32 masters."""

    def __init__(self, W1, b1, W2, b2, w3, b3):
        self.W1 = np.array(W1, np.float64)
        self.b1 = np.array(b1, np.float64)
        self.W2 = np.array(W2, np.float64)
        self.b2 = np.array(b2, np.float64)
        self.w3 = np.array(w3, np.float64)
        self.b3 = float(b3)

    def params(self):
        return dict(W1=self.W1, b1=self.b1, W2=self.W2, b2=self.b2, w3=self.w3, b3=np.array([self.b3]))

    def forward(self, X, round_bf16=True):
        r = bf16_round if round_bf16 else (lambda a: np.asarray(a, np.float64))
        W1 = r(self.W1)
        W2 = r(self.W2)
        A1 = r(np.maximum(X @ W1.T + self.b1, 0.0))
        A2 = r(np.maximum(A1 @ W2.T + self.b2, 0.0))
        y = A2 @ self.w3 + self.b3
        return dict(X=X, A1=A1, A2=A2, y=y, W1r=W1, W2r=W2)

    def loss(self, X, t, round_bf16=True):
        y = self.forward(X, round_bf16)["y"]
        return float(np.mean((y - t) ** 2))

    def backward(self, X, t, round_bf16=True):
        r = bf16_round if round_bf16 else (lambda a: np.asarray(a, np.float64))
        f = self.forward(X, round_bf16)
        B = X.shape[0]
        dy = 2.0 * (f["y"] - t) / B
        g = {}
        g["w3"] = f["A2"].T @ dy
        g["b3"] = np.array([dy.sum()])
        dZ2 = r(np.outer(dy, self.w3) * (f["A2"] > 0))
        g["W2"] = dZ2.T @ f["A1"]
        g["b2"] = dZ2.sum(0)
        dZ1 = r((dZ2 @ f["W2r"]) * (f["A1"] > 0))
        g["W1"] = dZ1.T @ X
        g["b1"] = dZ1.sum(0)
        return dict(loss=float(np.mean((f["y"] - t) ** 2)), y=f["y"], grads=g, dZ1=dZ1, dZ2=dZ2, A1=f["A1"],
                    A2=f["A2"])


def adam_step(p, g, m, v, k, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step number k >= 1) in float64; returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** k)
    vh = v / (1 - b2 ** k)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
