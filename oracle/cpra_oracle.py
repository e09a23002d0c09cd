"""FP64 CPU oracle for one CPRA training step (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The product path (the CUDA library and
its Python binding) never calls it and shares no code with it.

What it computes, in the paper's order and notation (Ichikawa & Iwashita,
"Continuous Parallel Relaxation for Finding Diverse Solutions in
Combinatorial Optimization Problems"):

  forward   Eq. GCN (App. B.1) twice, with the two-layer architecture of
            App. C.1: node embeddings h^0 (N x H0) -> conv -> ReLU -> conv
            (width S) -> sigmoid  =>  P in [0,1]^{N x S}.
  loss      Eq. (CPRA-loss-function-GNN-penalty) / (...-variation):
            R = sum_s l(P_:s; C, lambda_s) + gamma * S(P) + nu * Psi(P),
            S(P) = sum_{i,s} 1 - (2 P_is - 1)^alpha,
            Psi(P) = -S * sum_i STD_s[P_is]  (population STD, Notation sec.).
            l is the MIS or MaxCut QUBO of Table "objective-functions"
            (App. C.3) with x relaxed to P (Background, continuous relaxation).
  gradient  analytic chain rule through sigmoid, both GCN layers and the
            node embeddings (plain calculus; no autograd).
  update    Adam / AdamW (Implementation paragraph of the Experiments section).
  rounding  x_is = 1[P_is > 0.5] (App. C.2), integer MIS size / violations /
            MaxCut cut per shot, and the pairwise Hamming sum of Prop. 3.2.

Readings of points the paper leaves open:
  * annealing sign: S(P) = sum(1 - (2P-1)^alpha) with gamma increasing from
    negative (convex, P -> 1/2) to positive (binarising), per Theorem 3.1;
  * d/dp (1-(2p-1)^alpha) = -2 alpha (2p-1)^(alpha-1) (App. A prints the
    alpha = 2 case only);
  * every undirected edge counted once in the MIS penalty and the MaxCut sum;
  * Psi gradient is zero on rows whose variance across shots is exactly 0;
  * the ReLU sign is a discrete decision taken from floating point: for the
    BF16 form it is taken on bfloat16-rounded operands, as the kernels do
    (``relu_decision="bf16"``); every value stays float64;
  * the optional "VAR" diversity form Psi_var = -S^2 sum_i VAR_s[P_is] is the
    left-hand side of Prop. 3.2 (negated);
  * parameters: one self weight B^k, one neighbour weight W^k and one bias
    per layer (this reproduces the parameter counts printed in the tables of
    the Experiments section); the flat layout is
    [Wcat1 = [B1|W1] (H1 x 2H0), b1, Wcat2 = [B2|W2] (S x 2H1), b2];
  * node embeddings are trainable (h^0_{v,theta}, App. C.1) but are not
    counted as parameters by those tables.

Parity status: every function below is pinned by tests under tests/
(brute force, closed forms, invariants, finite differences, library
routines).  Multi-step trajectories are not pinned (the iteration is
chaotic); parity is per step from identical inputs.
"""
from __future__ import annotations

import numpy as np

MIS = 0
MAXCUT = 1
WMIS = 2   # weighted MIS (App. two-stage experiment): weight w_is of node i in task s
DBM = 3    # diverse bipartite matching (Eq. matching-cost-function), one instance per shot


def relu(x):
    return np.maximum(x, 0.0)


def dbm_parts(P, inst):
    """Row sums R (N1 x S), column sums K (N2 x S), totals T, U = sum M P and
    the matching reward sum C P per shot, for variables x_ij at node i*N2 + j."""
    N1, N2 = inst["N1"], inst["N2"]
    S = P.shape[1]
    X = P.reshape(N1, N2, S)
    C = np.asarray(inst["C"], np.float64).reshape(N1, N2, S)
    M = np.asarray(inst["M"], np.float64).reshape(N1, N2, S)
    return dict(R=X.sum(axis=1), K=X.sum(axis=0), T=X.sum(axis=(0, 1)),
                U=(M * X).sum(axis=(0, 1)), CP=(C * X).sum(axis=(0, 1)), C=C, M=M, X=X)


def dbm_penalty(parts, inst):
    """lambda-weighted penalty of Eq. matching-cost-function per shot."""
    lam4 = np.asarray(inst["lam4"], np.float64)          # S x 4
    pq = np.asarray(inst["pq"], np.float64)              # S x 2
    T, U = parts["T"], parts["U"]
    return (lam4[:, 0] * relu(parts["R"] - 1.0).sum(axis=0)
            + lam4[:, 1] * relu(parts["K"] - 1.0).sum(axis=0)
            + lam4[:, 2] * relu(pq[:, 0] * T - U)
            + lam4[:, 3] * relu(pq[:, 1] * T - (T - U)))
DIV_STD = 0
DIV_VAR = 1


# --------------------------------------------------------------------------
# graph helpers
# --------------------------------------------------------------------------
class Graph:
    """Symmetric CSR plus the undirected edge list (i < j), in float64."""

    def __init__(self, rowptr, col, weights=None):
        self.rowptr = np.asarray(rowptr, dtype=np.int64)
        self.col = np.asarray(col, dtype=np.int64)
        self.N = len(self.rowptr) - 1
        self.deg = np.diff(self.rowptr).astype(np.int64)
        rows = np.repeat(np.arange(self.N, dtype=np.int64), self.deg)
        self.rows = rows                       # source row of each CSR entry
        w = np.ones(len(self.col)) if weights is None else np.asarray(weights, np.float64)
        self.w_csr = w
        keep = rows < self.col
        self.ei = rows[keep]                   # undirected edges, each once
        self.ej = self.col[keep]
        self.ew = w[keep]
        # weighted degree sum_j A_ij (MaxCut linear term)
        self.wdeg = np.zeros(self.N)
        np.add.at(self.wdeg, rows, w)


def mean_aggregate(g: Graph, X: np.ndarray) -> np.ndarray:
    """a_v = (1/|N(v)|) sum_{u in N(v)} X_u  (Eq. GCN, App. B.1); 0 if isolated."""
    out = np.zeros((g.N, X.shape[1]))
    np.add.at(out, g.rows, X[g.col])
    nz = g.deg > 0
    out[nz] /= g.deg[nz, None]
    return out


def mean_aggregate_adjoint(g: Graph, Y: np.ndarray) -> np.ndarray:
    """Adjoint of mean_aggregate: out_u = sum_{v : u in N(v)} Y_v / |N(v)|.

    Written as the literal transpose: every CSR entry (v -> u) of row v sends
    Y_v / deg_v to u."""
    out = np.zeros((g.N, Y.shape[1]))
    scale = np.zeros(g.N)
    nz = g.deg > 0
    scale[nz] = 1.0 / g.deg[nz]
    np.add.at(out, g.col, Y[g.rows] * scale[g.rows, None])
    return out


# --------------------------------------------------------------------------
# parameters
# --------------------------------------------------------------------------
def param_count(H0: int, H1: int, S: int) -> int:
    """B1, W1 (H1 x H0 each), b1 (H1), B2, W2 (S x H1 each), b2 (S)."""
    return 2 * H1 * H0 + H1 + 2 * S * H1 + S


def unpack(theta: np.ndarray, H0: int, H1: int, S: int):
    theta = np.asarray(theta, dtype=np.float64)
    o = 0
    Wcat1 = theta[o:o + H1 * 2 * H0].reshape(H1, 2 * H0); o += H1 * 2 * H0
    b1 = theta[o:o + H1]; o += H1
    Wcat2 = theta[o:o + S * 2 * H1].reshape(S, 2 * H1); o += S * 2 * H1
    b2 = theta[o:o + S]; o += S
    assert o == len(theta), "theta has the wrong length"
    return dict(B1=Wcat1[:, :H0], W1=Wcat1[:, H0:], b1=b1,
                B2=Wcat2[:, :H1], W2=Wcat2[:, H1:], b2=b2)


def pack(B1, W1, b1, B2, W2, b2) -> np.ndarray:
    return np.concatenate([np.concatenate([B1, W1], axis=1).ravel(), b1,
                           np.concatenate([B2, W2], axis=1).ravel(), b2])


# --------------------------------------------------------------------------
# forward: two GCN layers (Eq. GCN), ReLU, sigmoid head of width S (App. C.1)
# --------------------------------------------------------------------------
def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def bf16_round(x) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float64.  bfloat16 keeps the float32 sign and exponent and the top 7
    mantissa bits."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(g: Graph, theta, X0, H0, H1, S, relu_decision=None, init_logits=None):
    """relu_decision: None decides the ReLU sign 1[Z1 > 0] on the float64
    Z1; "bf16" decides it on Z1 recomputed from bfloat16-rounded operands
    (X0, the neighbour mean and the weights), the precision in which the
    BF16 form's kernels take that decision.  All values stay float64.
    init_logits: optional N x S warm-start offset L0 added to the head's
    pre-activation (Z2 = ... + b2 + L0); constant, so the gradient formulas
    are unchanged."""
    p = unpack(theta, H0, H1, S)
    X0 = np.asarray(X0, dtype=np.float64)
    M1 = mean_aggregate(g, X0)
    Z1 = X0 @ p["B1"].T + M1 @ p["W1"].T + p["b1"]
    if relu_decision is None:
        on = Z1 > 0.0
    elif relu_decision == "bf16":
        xb = bf16_round(X0)
        mb = bf16_round(mean_aggregate(g, xb))
        zd = xb @ bf16_round(p["B1"]).T + mb @ bf16_round(p["W1"]).T + p["b1"]
        on = zd > 0.0
    else:
        raise ValueError("relu_decision")
    H1a = np.where(on, Z1, 0.0)
    M2 = mean_aggregate(g, H1a)
    Z2 = H1a @ p["B2"].T + M2 @ p["W2"].T + p["b2"]
    if init_logits is not None:
        Z2 = Z2 + np.asarray(init_logits, dtype=np.float64)
    P = sigmoid(Z2)
    return dict(X0=X0, M1=M1, Z1=Z1, relu_on=on, H1=H1a, M2=M2, Z2=Z2, P=P)


# --------------------------------------------------------------------------
# relaxed loss terms (Eq. CPRA-loss-function-GNN, -penalty, -variation)
# --------------------------------------------------------------------------
def shot_variance(P: np.ndarray) -> np.ndarray:
    """VAR_s[P_is] per node i, population form (Notation section)."""
    S = P.shape[1]
    m = P.sum(axis=1) / S
    return ((P - m[:, None]) ** 2).sum(axis=1) / S


def loss_terms(g: Graph, P, lam, problem, alpha, div_kind=DIV_STD, weights=None, inst=None):
    """Per-shot cost_s, pen_s, ann_s and the shot-coupling Psi.

    MIS    l = -sum_i p_i + lambda sum_{(i,j) in E} p_i p_j
           cost_s = -sum_i P_is, pen_s = sum_{(i,j) in E} P_is P_js
    MaxCut l = sum_{i<j} A_ij (2 p_i p_j - p_i - p_j); cost_s = l, pen_s = 0
    WMIS   l = -sum_i w_i p_i + lambda sum_{(i,j) in E} p_i p_j (task s has its
           own node weights w_:s); cost_s = -sum_i w_is P_is, pen_s as MIS
    DBM    Eq. matching-cost-function on x_ij = P_{i*N2+j}, instance (C, M,
           lambda_1..4, p, q) of shot s in `inst`; cost_s = -sum C P and
           pen_s = the four lambda-weighted ReLU terms (so l = cost + pen)
    ann_s  = sum_i 1 - (2 P_is - 1)^alpha
    Psi    = -S sum_i STD_s[P_is]        (STD form, Eq. ...-variation)
           = -S^2 sum_i VAR_s[P_is]      (VAR form, Prop. 3.2 left-hand side)
    """
    P = np.asarray(P, dtype=np.float64)
    S = P.shape[1]
    Pi, Pj = P[g.ei], P[g.ej]
    if problem == MIS:
        cost = -P.sum(axis=0)
        pen = (Pi * Pj).sum(axis=0)
    elif problem == WMIS:
        cost = -(np.asarray(weights, dtype=np.float64) * P).sum(axis=0)
        pen = (Pi * Pj).sum(axis=0)
    elif problem == DBM:
        parts = dbm_parts(P, inst)
        cost = -parts["CP"]
        pen = dbm_penalty(parts, inst)
    elif problem == MAXCUT:
        cost = (g.ew[:, None] * (2.0 * Pi * Pj - Pi - Pj)).sum(axis=0)
        pen = np.zeros(S)
    else:
        raise ValueError("problem")
    ann = (1.0 - (2.0 * P - 1.0) ** alpha).sum(axis=0)
    var = shot_variance(P)
    if div_kind == DIV_STD:
        psi = -S * np.sqrt(var).sum()
    elif div_kind == DIV_VAR:
        psi = -(S ** 2) * var.sum()
    else:
        raise ValueError("div_kind")
    return dict(cost=cost, pen=pen, ann=ann, psi=psi)


def total_loss(terms, lam, gamma, nu, problem):
    lam = np.asarray(lam, dtype=np.float64)
    base = terms["cost"].sum()
    if problem == DBM:
        base += terms["pen"].sum()            # already lambda-weighted
    elif problem in (MIS, WMIS):
        base += (lam * terms["pen"]).sum()
    return base + gamma * terms["ann"].sum() + nu * terms["psi"]


def grad_P(g: Graph, P, lam, problem, alpha, gamma, nu, div_kind=DIV_STD, weights=None,
           inst=None):
    """dR/dP_is, analytic, with the edge list traversed once per edge."""
    P = np.asarray(P, dtype=np.float64)
    N, S = P.shape
    G = np.zeros((N, S))
    if problem in (MIS, WMIS):
        lam = np.asarray(lam, dtype=np.float64)
        G -= 1.0 if problem == MIS else np.asarray(weights, dtype=np.float64)
        np.add.at(G, g.ei, lam[None, :] * P[g.ej])
        np.add.at(G, g.ej, lam[None, :] * P[g.ei])
    elif problem == DBM:
        # d/dx_ij of Eq. matching-cost-function, ReLU'(0) = 0
        parts = dbm_parts(P, inst)
        lam4 = np.asarray(inst["lam4"], np.float64)
        pq = np.asarray(inst["pq"], np.float64)
        T, U = parts["T"], parts["U"]
        N1, N2 = inst["N1"], inst["N2"]
        rows = (parts["R"] > 1.0).astype(np.float64)        # N1 x S
        cols = (parts["K"] > 1.0).astype(np.float64)        # N2 x S
        on3 = (pq[:, 0] * T - U > 0.0).astype(np.float64)
        on4 = (pq[:, 1] * T - (T - U) > 0.0).astype(np.float64)
        Gd = (-parts["C"] + lam4[:, 0] * rows[:, None, :] + lam4[:, 1] * cols[None, :, :]
              + lam4[:, 2] * on3 * (pq[:, 0] - parts["M"])
              + lam4[:, 3] * on4 * (pq[:, 1] - (1.0 - parts["M"])))
        G += Gd.reshape(N1 * N2, S)
    else:
        w = g.ew[:, None]
        np.add.at(G, g.ei, w * (2.0 * P[g.ej] - 1.0))
        np.add.at(G, g.ej, w * (2.0 * P[g.ei] - 1.0))
    # gamma * d/dp [1 - (2p-1)^alpha] = -2 alpha gamma (2p-1)^(alpha-1)
    G += -2.0 * alpha * gamma * (2.0 * P - 1.0) ** (alpha - 1)
    if nu != 0.0:
        m = P.sum(axis=1) / S
        dev = P - m[:, None]
        var = (dev ** 2).sum(axis=1) / S
        if div_kind == DIV_STD:
            # d/dP_is [-S sqrt(VAR_i)] = -(P_is - m_i) / sqrt(VAR_i)
            gd = np.zeros_like(P)
            nz = var > 0.0
            gd[nz] = -dev[nz] / np.sqrt(var[nz])[:, None]
        else:
            # d/dP_is [-S^2 VAR_i] = -2 S (P_is - m_i)
            gd = -2.0 * S * dev
        G += nu * gd
    return G


# --------------------------------------------------------------------------
# backward through the GNN (chain rule of Eq. GCN twice)
# --------------------------------------------------------------------------
def backward(g: Graph, theta, cache, G_P, H0, H1, S):
    p = unpack(theta, H0, H1, S)
    P = cache["P"]
    G_Z2 = G_P * P * (1.0 - P)                    # sigmoid'
    dB2 = G_Z2.T @ cache["H1"]
    dW2 = G_Z2.T @ cache["M2"]
    db2 = G_Z2.sum(axis=0)
    G_H1 = G_Z2 @ p["B2"] + mean_aggregate_adjoint(g, G_Z2 @ p["W2"])
    G_Z1 = G_H1 * cache["relu_on"]                # ReLU'
    dB1 = G_Z1.T @ cache["X0"]
    dW1 = G_Z1.T @ cache["M1"]
    db1 = G_Z1.sum(axis=0)
    G_X0 = G_Z1 @ p["B1"] + mean_aggregate_adjoint(g, G_Z1 @ p["W1"])
    return dict(theta=pack(dB1, dW1, db1, dB2, dW2, db2), X0=G_X0,
                G_Z2=G_Z2, G_Z1=G_Z1)


# --------------------------------------------------------------------------
# optimiser and annealing schedule
# --------------------------------------------------------------------------
def adam(theta, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One Adam step (Kingma & Ba), t >= 1; wd > 0 adds AdamW's decoupled
    decay theta <- theta (1 - lr wd) before the moment step."""
    theta = np.asarray(theta, np.float64)
    m = np.asarray(m, np.float64)
    v = np.asarray(v, np.float64)
    grad = np.asarray(grad, np.float64)
    if wd != 0.0:
        theta = theta * (1.0 - lr * wd)
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    theta = theta - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v


def gamma_schedule(t, T, gamma0, gamma1):
    """Linear anneal gamma_t = gamma0 + (gamma1 - gamma0) t / (T - 1)."""
    if T <= 1:
        return gamma1
    return gamma0 + (gamma1 - gamma0) * min(t, T - 1) / (T - 1)


def early_stop_step(terms_seq, gammas, lam, problem, tol, patience, ann_below=0.0):
    """Early stopping of the Implementation paragraph: the run is monitored
    through the summed penalty-form loss l_t = sum_s (cost_s + lambda_s pen_s)
    (MaxCut: sum_s cost_s; DBM: sum_s (cost_s + pen_s)) and the annealing term phi_t = gamma_t sum_s ann_s,
    with a tolerance and a patience.  Reading (the paper gives only the two
    numbers): step t > 0 is stale when, for both monitored values, the change
    from step t-1 is positive or at most `tol` in magnitude; the run stops at
    the step that completes `patience` consecutive stale steps.  Sums run over
    s = 0..S-1 in order, in float64, from the per-step terms as given.

    With ann_below > 0, a step whose annealing sum sum_s ann_s is below it
    stops the run as well (the stopping rule of the two-stage experiment,
    App. two-stage); patience 0 disables the stale-step rule.

    terms_seq: per step (cost[S], pen[S], ann[S]); gammas: per step gamma_t.
    Returns the index of the stopping step, or -1."""
    prev = None
    count = 0
    for t, ((cost, pen, ann), gamma) in enumerate(zip(terms_seq, gammas)):
        l_t = 0.0
        a_t = 0.0
        for s in range(len(cost)):
            ls = float(cost[s])
            if problem in (MIS, WMIS):
                ls = ls + float(lam[s]) * float(pen[s])
            elif problem == DBM:
                ls = ls + float(pen[s])          # the DBM penalty carries its own lambdas
            l_t = l_t + ls
            a_t = a_t + float(ann[s])
        phi_t = float(gamma) * a_t
        if ann_below > 0.0 and a_t < ann_below:
            return t
        if patience > 0 and prev is not None:
            dl = l_t - prev[0]
            dp = phi_t - prev[1]
            stale = (dl > 0.0 or abs(dl) <= tol) and (dp > 0.0 or abs(dp) <= tol)
            count = count + 1 if stale else 0
            if count >= patience:
                return t
        prev = (l_t, phi_t)
    return -1


# --------------------------------------------------------------------------
# rounding and integer evaluation (App. C.2, Table objective-functions)
# --------------------------------------------------------------------------
def round_solutions(P) -> np.ndarray:
    """x_is = 0 if P_is <= 0.5 else 1."""
    return (np.asarray(P) > 0.5).astype(np.int64)


def integer_eval(g: Graph, X, lam, problem, weights=None, inst=None):
    """Per shot: objective (MIS set size / MaxCut cut size), violations
    (MIS: edges with both ends selected; MaxCut: 0), qubo value l(x), the
    objective in the problem's own units `value` (set size, total weight of
    the set for weighted MIS, cut weight sum_{cut edges} A_ij for MaxCut --
    the cut size with unit weights), and the pairwise Hamming sum
    sum_{s<l} d_H(x_s, x_l).  DBM: objective = matched pairs sum x, violations =
    rows and columns with more than one pair plus the two diversity
    constraints that fail, value = sum C x, qubo = l(x)."""
    X = np.asarray(X, dtype=np.int64)
    N, S = X.shape
    Xi, Xj = X[g.ei], X[g.ej]
    if problem == DBM:
        parts = dbm_parts(X.astype(np.float64), inst)
        pq = np.asarray(inst["pq"], np.float64)
        T, U = parts["T"], parts["U"]
        obj = X.sum(axis=0)
        viol = ((parts["R"] > 1.0).sum(axis=0) + (parts["K"] > 1.0).sum(axis=0)
                + (pq[:, 0] * T - U > 0.0) + (pq[:, 1] * T - (T - U) > 0.0))
        value = parts["CP"]
        qubo = -value + dbm_penalty(parts, inst)
    elif problem in (MIS, WMIS):
        obj = X.sum(axis=0)
        viol = (Xi * Xj).sum(axis=0)
        value = obj.astype(np.float64)
        if problem == WMIS:
            value = (np.asarray(weights, dtype=np.float64) * X).sum(axis=0)
        qubo = -value + np.asarray(lam, np.float64) * viol
    else:
        obj = (Xi != Xj).sum(axis=0)
        viol = np.zeros(S, dtype=np.int64)
        value = (g.ew[:, None] * (Xi != Xj)).sum(axis=0)   # the (weighted) cut
        qubo = -value
    k = X.sum(axis=1)
    pair_hamming = int((k * (S - k)).sum())
    return dict(objective=obj.astype(np.int64), violations=viol.astype(np.int64),
                qubo=qubo.astype(np.float64), value=np.asarray(value, np.float64),
                pair_hamming=pair_hamming)


def pack_bits(X) -> np.ndarray:
    """Rounded solutions as uint32 words: bit (s mod 32) of word s // 32 of
    row i is x_is.  Shape N x ceil(S/32)."""
    X = np.asarray(X, dtype=np.uint64)
    N, S = X.shape
    W = (S + 31) // 32
    out = np.zeros((N, W), dtype=np.uint64)
    for s in range(S):
        out[:, s // 32] |= X[:, s] << np.uint64(s % 32)
    return out.astype(np.uint32)


# --------------------------------------------------------------------------
# one full training step
# --------------------------------------------------------------------------
def step(g: Graph, theta, X0, cfg, t, adam_state=None):
    """One CPRA step at iteration t (1-based for Adam bias correction).

    cfg keys: H0, H1, S, problem, alpha, lam (S), gamma, nu, div_kind,
    lr, beta1, beta2, eps, wd, train_embedding, optional weights (N x S,
    weighted MIS) and train_encoder (False: only the head Wcat2, b2 is
    updated, as in the fine-tuning stage of the two-stage schedule).
    adam_state: dict(m_theta, v_theta, m_X0, v_X0) or None (zeros)."""
    H0, H1, S = cfg["H0"], cfg["H1"], cfg["S"]
    cache = forward(g, theta, X0, H0, H1, S, cfg.get("relu_decision"), cfg.get("init_logits"))
    P = cache["P"]
    W = cfg.get("weights")
    inst = cfg.get("dbm")
    terms = loss_terms(g, P, cfg["lam"], cfg["problem"], cfg["alpha"], cfg["div_kind"], W, inst)
    L = total_loss(terms, cfg["lam"], cfg["gamma"], cfg["nu"], cfg["problem"])
    G_P = grad_P(g, P, cfg["lam"], cfg["problem"], cfg["alpha"], cfg["gamma"],
                 cfg["nu"], cfg["div_kind"], W, inst)
    grads = backward(g, theta, cache, G_P, H0, H1, S)
    if adam_state is None:
        adam_state = dict(m_theta=np.zeros(len(theta)), v_theta=np.zeros(len(theta)),
                          m_X0=np.zeros(np.shape(X0)), v_X0=np.zeros(np.shape(X0)))
    hp = dict(lr=cfg["lr"], beta1=cfg["beta1"], beta2=cfg["beta2"], eps=cfg["eps"],
              wd=cfg["wd"])
    th1, mt, vt = adam(theta, adam_state["m_theta"], adam_state["v_theta"],
                       grads["theta"], t, **hp)
    encoder = cfg.get("train_encoder", True)
    if not encoder:  # head only: layer-1 weights and the embeddings keep their values
        h0 = 2 * H1 * H0 + H1
        th1[:h0] = np.asarray(theta, np.float64)[:h0]
        mt[:h0] = np.asarray(adam_state["m_theta"], np.float64)[:h0]
        vt[:h0] = np.asarray(adam_state["v_theta"], np.float64)[:h0]
    if cfg.get("train_embedding", True) and encoder:
        x1, mx, vx = adam(X0, adam_state["m_X0"], adam_state["v_X0"], grads["X0"], t, **hp)
    else:
        x1 = np.asarray(X0, np.float64)
        mx = np.asarray(adam_state["m_X0"], np.float64)
        vx = np.asarray(adam_state["v_X0"], np.float64)
    X = round_solutions(P)
    ev = integer_eval(g, X, cfg["lam"], cfg["problem"], W, inst)
    return dict(cache=cache, P=P, terms=terms, loss=L, G_P=G_P, grads=grads,
                theta_next=th1, X0_next=x1,
                adam_next=dict(m_theta=mt, v_theta=vt, m_X0=mx, v_X0=vx),
                X=X, eval=ev)
