"""Pins of the warm-start network's FP64 oracle (three Eq. GCN layers fitted
with the mean binary cross-entropy)."""
import numpy as np
import pytest

from oracle import cpra_oracle as O
from oracle import warm_oracle as WO
from paper_2402_02190_gb300 import inputs as I


def _small(F=4, H=5, S=3, N=14, seed=0):
    rp, col = I.erdos_renyi_graph(N, 0.3, seed=seed)
    g = O.Graph(rp, col)
    rng = np.random.default_rng(seed)
    theta = rng.normal(size=WO.param_count(F, H, S)) * 0.7
    X = rng.normal(size=(N, F))
    Y = (rng.random((N, S)) < 0.4).astype(np.float64)
    return g, theta, X, Y


def test_param_count_and_layout():
    assert WO.param_count(16, 64, 32) == I.ws_param_count(16, 64, 32) == 2 * 64 * 16 + 64 + 2 * 64 * 64 + 64 + 2 * 32 * 64 + 32
    th = np.arange(WO.param_count(2, 3, 4), dtype=np.float64)
    p = WO.unpack(th, 2, 3, 4)
    assert np.array_equal(WO.pack(p["W1"], p["b1"], p["W2"], p["b2"], p["W3"], p["b3"]), th)
    assert p["W3"].shape == (4, 6) and p["b3"][0] == th[-4]


def test_cross_entropy_closed_forms():
    # logits 0: log 2 whatever the target; large logits of the right sign: ~0
    assert WO.bce(np.zeros((3, 2)), np.array([[0, 1], [1, 1], [0, 0]])) == pytest.approx(np.log(2.0))
    assert WO.bce(np.array([[40.0, -40.0]]), np.array([[1, 0]])) < 1e-15
    # softplus(z) - y z equals -log sigmoid(z) for y = 1 and -log(1 - sigmoid(z)) for y = 0
    z = np.array([[-3.0, 0.5, 7.0]])
    s = 1 / (1 + np.exp(-z))
    assert WO.bce(z, np.ones_like(z)) == pytest.approx(np.mean(-np.log(s)), rel=1e-14)
    assert WO.bce(z, np.zeros_like(z)) == pytest.approx(np.mean(-np.log(1 - s)), rel=1e-14)


def test_without_neighbour_weights_is_a_per_node_mlp():
    F, H, S = 4, 5, 3
    g, theta, X, _ = _small(F, H, S)
    p = WO.unpack(theta, F, H, S)
    W1, W2, W3 = p["W1"].copy(), p["W2"].copy(), p["W3"].copy()
    W1[:, F:] = 0
    W2[:, H:] = 0
    W3[:, H:] = 0
    th = WO.pack(W1, p["b1"], W2, p["b2"], W3, p["b3"])
    Z3 = WO.forward(g, th, X, F, H, S)["Z3"]
    h1 = np.maximum(X @ W1[:, :F].T + p["b1"], 0)
    h2 = np.maximum(h1 @ W2[:, :H].T + p["b2"], 0)
    assert np.allclose(Z3, h2 @ W3[:, :H].T + p["b3"], rtol=0, atol=1e-13)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_finite_differences(seed):
    F, H, S = 4, 5, 3
    g, theta, X, Y = _small(F, H, S, seed=seed)
    c = WO.forward(g, theta, X, F, H, S)
    grad = WO.backward(g, theta, c, Y, F, H, S)

    def L(th):
        return WO.bce(WO.forward(g, th, X, F, H, S)["Z3"], Y)

    h = 1e-6
    fd = np.empty_like(theta)
    for k in range(theta.size):
        e = np.zeros_like(theta)
        e[k] = h
        fd[k] = (L(theta + e) - L(theta - e)) / (2 * h)
    assert np.allclose(grad, fd, rtol=1e-5, atol=1e-9)


def test_bf16_relu_decision_only_moves_the_mask():
    F, H, S = 4, 5, 3
    g, theta, X, _ = _small(F, H, S)
    a = WO.forward(g, theta, X, F, H, S)
    b = WO.forward(g, theta, X, F, H, S, relu_decision="bf16")
    # the decisions can differ only where the pre-activation is tiny
    d1 = a["on1"] != b["on1"]
    assert np.all(np.abs(a["Z1"][d1]) < 0.05)
    assert np.array_equal(a["Z1"], b["Z1"])


def test_bf16_layer1_decision_flips_only_within_the_rounding_bound():
    """Layer 1 of the warm network under the BF16 reading: its ReLU sign may
    only differ from the FP64 sign where |Z1| is within the worst-case error
    that bfloat16 rounding (through float32: u = 2^-8 + 2^-22 relative) of X,
    of the neighbour mean of the rounded rows and of W1 can put into Z1;
    a decision taken on a wrong operand or without the bias would flip signs
    outside that bound."""
    F, H, S, N = 16, 32, 8, 600
    rp, col = I.random_regular_graph(N, 5, 3)
    g = O.Graph(rp, col)
    rng = np.random.default_rng(4)
    theta = rng.normal(size=WO.param_count(F, H, S)) * 0.3
    X = rng.normal(size=(N, F))
    a = WO.forward(g, theta, X, F, H, S)
    b = WO.forward(g, theta, X, F, H, S, relu_decision="bf16")
    W1 = np.abs(WO.unpack(theta, F, H, S)["W1"])          # H x 2F, [self | neighbour]
    u = 2.0 ** -8 + 2.0 ** -22
    mb = O.mean_aggregate(g, O.bf16_round(X))
    dA = np.concatenate([u * np.abs(X),
                         u * O.mean_aggregate(g, np.abs(X)) + u * np.abs(mb)], axis=1)
    E0 = np.concatenate([np.abs(O.bf16_round(X)), np.abs(O.bf16_round(mb))], axis=1)
    bound = (dA @ W1.T + E0 @ (u * W1).T) * (1 + 1e-9) + 1e-300
    flipped = a["on1"] != b["on1"]
    assert flipped.sum() > 0
    assert np.all(np.abs(a["Z1"][flipped]) <= bound[flipped])
    assert (np.abs(a["Z1"]) <= bound).mean() < 0.05
