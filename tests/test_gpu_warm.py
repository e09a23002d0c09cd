"""Warm-start network on the GPU (cpra_ws_*): one training step and the
forward against the FP64 oracle, the device feature generator's properties,
and the warm-start offset carried into a CPRA run."""
import numpy as np
import pytest

from oracle import cpra_oracle as O
from oracle import warm_oracle as WO
from paper_2402_02190_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2402_02190_gb300 import cpra  # noqa: E402


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _case(precision, N, d, F, H, S, seed):
    rp, col = I.random_regular_graph(N, d, seed)
    X = I.seeded_ws_features(rp, F, seed + 1)
    bits = I.seeded_bits(N, S, seed + 2)
    theta = I.seeded_ws_params(F, H, S, seed + 3, scale=1.5)
    net = cpra.WarmStartNet(N, len(col), F=F, H=H, S=S, precision=precision, lr=1e-3)
    net.set_params(theta)
    t = dict(rp=_dev(rp.astype(np.int32)), col=_dev(col.astype(np.int32)), X=_dev(X),
             bits=_dev(bits.view(np.int32)))
    return rp, col, X, bits, theta, net, t


@pytest.mark.parametrize("precision,tol", [(cpra.FP32, 1e-5), (cpra.BF16, 2e-2)])
@pytest.mark.parametrize("shape", [(500, 4, 16, 32, 20), (1200, 3, 32, 64, 32), (334, 5, 16, 48, 7)])
def test_train_step_matches_oracle(precision, tol, shape):
    N, d, F, H, S = shape
    rp, col, X, bits, theta, net, t = _case(precision, N, d, F, H, S, seed=N)
    g = O.Graph(rp, col)
    Y = I.unpack_bits(bits, S).astype(np.float64)
    c = WO.forward(g, theta, X, F, H, S, relu_decision="bf16" if precision == cpra.BF16 else None)
    logits = net.predict(t["rp"], t["col"], t["X"]).cpu().numpy().astype(np.float64)
    err = np.abs(logits - c["Z3"]).max() / np.abs(c["Z3"]).max()
    assert err <= tol, err
    loss = net.train_step(t["rp"], t["col"], t["X"], t["bits"])
    L = WO.bce(c["Z3"], Y)
    assert abs(loss - L) <= tol * L
    grad = net.params(1).astype(np.float64)
    gref = WO.backward(g, theta, c, Y, F, H, S)
    o = 0
    for n in (2 * H * F, H, 2 * H * H, H, 2 * S * H, S):
        e = np.linalg.norm(grad[o:o + n] - gref[o:o + n]) / np.linalg.norm(gref[o:o + n])
        assert e <= tol, (o, n, e)
        o += n
    th_ref, _, _ = O.adam(theta.astype(np.float64), np.zeros(theta.size), np.zeros(theta.size),
                          gref, 1, 1e-3)
    step = np.linalg.norm(th_ref - theta)
    assert np.linalg.norm(net.params(0) - th_ref) <= 10 * tol * step
    net.close()
    if precision == cpra.BF16:
        # against the plain FP64 oracle (ReLU signs decided on FP64 values):
        # the logits, the loss and the last layer's gradient are continuous
        # where a sign flips and meet the same bar; the gradients of the
        # two ReLU layers are reported
        cp = WO.forward(g, theta, X, F, H, S)
        gp = WO.backward(g, theta, cp, Y, F, H, S)
        e_p = {"Z3": float(np.abs(logits - cp["Z3"]).max() / np.abs(cp["Z3"]).max()),
               "loss": float(abs(loss - WO.bce(cp["Z3"], Y)) / WO.bce(cp["Z3"], Y))}
        o = 0
        for name, n in (("W1", 2 * H * F), ("b1", H), ("W2", 2 * H * H), ("b2", H),
                        ("W3", 2 * S * H), ("b3", S)):
            e_p[name] = float(np.linalg.norm(grad[o:o + n] - gp[o:o + n]) / np.linalg.norm(gp[o:o + n]))
            o += n
        _report_plain(shape, e_p)
        for k in ("Z3", "loss", "W3", "b3"):
            assert e_p[k] <= tol, (k, e_p[k])


def _report_plain(shape, e_plain):
    """One JSON line per case to $CPRA_PARITY_REPORT (if set)."""
    import json
    import os
    path = os.environ.get("CPRA_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": "warm_train_step_bf16", "case": list(shape),
                                "vs_plain_fp64": e_plain}) + "\n")


def test_device_features():
    rp, col = I.random_regular_graph(20000, 5, seed=3)
    rpd = _dev(rp.astype(np.int32))
    net = cpra.WarmStartNet(20000, len(col), F=16, H=32, S=8)
    a = net.features(rpd, 7).cpu().numpy()
    b = net.features(rpd, 7).cpu().numpy()
    c = net.features(rpd, 8).cpu().numpy()
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.all(a[:, 0] == 1.0)
    assert np.array_equal(a[:, 1], (np.diff(rp) / 8.0).astype(np.float32))
    z = a[:, 2:]
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    net.close()


def test_training_reduces_the_loss_and_predictions_seed_cpra():
    """A few hundred steps on one graph fit its targets better than chance,
    and the logits, set as the CPRA head's offset, start P at sigmoid(L0)
    (the CPRA network's own output is small at initialisation)."""
    N, S = 2000, 16
    rp, col = I.random_regular_graph(N, 3, seed=9)
    bits = I.seeded_bits(N, S, 10, p=0.2)
    rpd, cold = _dev(rp.astype(np.int32)), _dev(col.astype(np.int32))
    net = cpra.WarmStartNet(N, len(col), F=16, H=64, S=S, lr=3e-3)
    X = net.features(rpd, 1)
    bd = _dev(bits.view(np.int32))
    first = net.train_step(rpd, cold, X, bd)
    for _ in range(300):
        last = net.train_step(rpd, cold, X, bd, want_loss=False)
    last = net.train_step(rpd, cold, X, bd)
    assert last < first
    L0 = net.predict(rpd, cold, X)
    lam = I.lambda_linspace(1, 4, S)
    s = cpra.Solver(rp, col, lam=lam, problem=cpra.MIS, S=S, H0=16, H1=16, precision=cpra.BF16)
    s.set_init_logits(L0)
    s.round_eval()  # a forward with the offset
    P = s.P()
    ref = 1.0 / (1.0 + np.exp(-L0.cpu().numpy().astype(np.float64)))
    # the GCN's own logits are small at initialisation but not zero
    assert np.corrcoef(P.ravel(), ref.ravel())[0, 1] > 0.9
    s.close()
    net.close()
