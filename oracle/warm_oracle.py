"""FP64 CPU oracle for the warm-start network (TEST INFRASTRUCTURE ONLY).

Only ``tests/`` may import this module; the product path never calls it.

The network is three layers of the paper's Eq. GCN (App. B.1): layer k maps
H_{k-1} to Z_k = H_{k-1} B_k^T + (D^-1 A H_{k-1}) W_k^T + b_k, with ReLU
after layers 1 and 2 and the logits Z_3 as output (S per node).  It is fitted
with the mean binary cross-entropy
    L = 1/(N S) sum_{i,s} softplus(Z3_is) - y_is Z3_is
against 0/1 targets y (rounded CPRA solutions).  Gradients are the plain
chain rule, written out; the optimiser is the same Adam as the CPRA step
(``cpra_oracle.adam``).  Flat parameter layout:
    [Wcat1 = [B1|W1] (H x 2F), b1 (H), Wcat2 (H x 2H), b2 (H),
     Wcat3 (S x 2H), b3 (S)].

Readings: the ReLU sign for the BF16 form is decided from bfloat16-rounded
operands of every layer (``relu_decision="bf16"``), as for the CPRA oracle;
values stay float64.

Parity status: pinned by tests/test_warm_oracle.py (closed forms of the
cross-entropy, the per-node-MLP special case, finite differences of every
gradient).
"""
from __future__ import annotations

import numpy as np

from oracle.cpra_oracle import Graph, bf16_round, mean_aggregate, mean_aggregate_adjoint


def param_count(F: int, H: int, S: int) -> int:
    return 2 * H * F + H + 2 * H * H + H + 2 * S * H + S


def unpack(theta, F, H, S):
    th = np.asarray(theta, dtype=np.float64)
    o = 0
    out = {}
    for name, shape in (("W1", (H, 2 * F)), ("b1", (H,)), ("W2", (H, 2 * H)), ("b2", (H,)),
                        ("W3", (S, 2 * H)), ("b3", (S,))):
        n = int(np.prod(shape))
        out[name] = th[o:o + n].reshape(shape)
        o += n
    assert o == th.size
    return out


def pack(W1, b1, W2, b2, W3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, np.ravel(W3), b3])


def forward(g: Graph, theta, X, F, H, S, relu_decision=None):
    p = unpack(theta, F, H, S)
    X = np.asarray(X, dtype=np.float64)
    A0 = np.concatenate([X, mean_aggregate(g, X)], axis=1)
    Z1 = A0 @ p["W1"].T + p["b1"]
    if relu_decision == "bf16":
        e0 = bf16_round(X)
        E0 = np.concatenate([e0, bf16_round(mean_aggregate(g, e0))], axis=1)
        z1d = E0 @ bf16_round(p["W1"]).T + p["b1"]
        on1 = z1d > 0.0
        e1 = bf16_round(np.where(on1, z1d, 0.0))
        E1 = np.concatenate([e1, bf16_round(mean_aggregate(g, e1))], axis=1)
        z2d = E1 @ bf16_round(p["W2"]).T + p["b2"]
    elif relu_decision is None:
        on1 = Z1 > 0.0
    else:
        raise ValueError("relu_decision")
    H1 = np.where(on1, Z1, 0.0)
    A1 = np.concatenate([H1, mean_aggregate(g, H1)], axis=1)
    Z2 = A1 @ p["W2"].T + p["b2"]
    on2 = (z2d > 0.0) if relu_decision == "bf16" else (Z2 > 0.0)
    H2 = np.where(on2, Z2, 0.0)
    A2 = np.concatenate([H2, mean_aggregate(g, H2)], axis=1)
    Z3 = A2 @ p["W3"].T + p["b3"]
    return dict(A0=A0, Z1=Z1, on1=on1, A1=A1, Z2=Z2, on2=on2, A2=A2, Z3=Z3)


def softplus(z):
    z = np.asarray(z, dtype=np.float64)
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def bce(Z3, Y) -> float:
    """Mean binary cross-entropy of logits Z3 against 0/1 targets Y."""
    Y = np.asarray(Y, dtype=np.float64)
    return float(np.mean(softplus(Z3) - Y * Z3))


def backward(g: Graph, theta, cache, Y, F, H, S):
    """Gradient of the mean cross-entropy with respect to the flat parameters."""
    p = unpack(theta, F, H, S)
    N = cache["Z3"].shape[0]
    Y = np.asarray(Y, dtype=np.float64)
    G3 = (1.0 / (1.0 + np.exp(-cache["Z3"])) - Y) / (N * S)
    dW3 = G3.T @ cache["A2"]
    db3 = G3.sum(axis=0)
    GA2 = G3 @ p["W3"]
    GZ2 = (GA2[:, :H] + mean_aggregate_adjoint(g, GA2[:, H:])) * cache["on2"]
    dW2 = GZ2.T @ cache["A1"]
    db2 = GZ2.sum(axis=0)
    GA1 = GZ2 @ p["W2"]
    GZ1 = (GA1[:, :H] + mean_aggregate_adjoint(g, GA1[:, H:])) * cache["on1"]
    dW1 = GZ1.T @ cache["A0"]
    db1 = GZ1.sum(axis=0)
    return pack(dW1, db1, dW2, db2, dW3, db3)
