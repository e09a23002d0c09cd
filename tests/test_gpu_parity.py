"""GPU parity tests: the CUDA path (through the C ABI) against the FP64 oracle
on identical seeded inputs.

Bars (from the method's precision split): FP32 form within 1e-5 relative,
BF16 dense layers within 2e-2 relative, rounding / integer objectives
bit-exact.  Loss terms use the cancellation-safe normaliser
|cost_s| + lambda_s |pen_s| + |gamma| ann_s per shot.
"""
import numpy as np
import pytest

from oracle import cpra_oracle as O
from oracle import exact as X
from paper_2402_02190_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2402_02190_gb300 import cpra  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    cpra.lib()


def rup(v, m):
    return (v + m - 1) // m * m


def dev_csr(rp, col):
    return (torch.tensor(rp.astype(np.int32), device="cuda"),
            torch.tensor(col.astype(np.int32), device="cuda"))


def graph_of(kind, N, seed):
    if kind[0] == "rrg":
        return I.random_regular_graph(N, kind[1], seed)
    return I.erdos_renyi_graph(N, kind[1] / (N - 1), seed)


def unpack_bits(bits, S):
    N = bits.shape[0]
    x = np.zeros((N, S), dtype=np.int64)
    for s in range(S):
        x[:, s] = (bits[:, s // 32] >> (s % 32)) & 1
    return x


# ===================================================================== loss
LOSS_CASES = [
    # problem, div, alpha, S, N, graph
    (O.MIS, O.DIV_STD, 2, 8, 1000, ("rrg", 3)),
    (O.MIS, O.DIV_VAR, 4, 100, 2000, ("rrg", 20)),
    (O.MAXCUT, O.DIV_STD, 2, 64, 3001, ("er", 10)),
    (O.MAXCUT, O.DIV_VAR, 2, 256, 1500, ("rrg", 5)),
    (O.MIS, O.DIV_STD, 2, 33, 777, ("er", 4)),
    (O.MIS, O.DIV_STD, 6, 1000, 300, ("rrg", 3)),
    (O.MAXCUT, O.DIV_STD, 2, 1, 500, ("rrg", 3)),
]


@pytest.mark.parametrize("grad_kind", [0, 1])
@pytest.mark.parametrize("case", LOSS_CASES)
def test_op_loss_matches_oracle(case, grad_kind):
    problem, div, alpha, S, N, gk = case
    rp, col = graph_of(gk, N, seed=S + N)
    g = O.Graph(rp, col)
    P = I.seeded_P(N, S, seed=N)
    lam = I.lambda_geomspace(0.5, 10.0, S)
    gamma, nu = -0.8, 0.37
    ld = rup(S, 16)
    Pd = torch.full((N, ld), 0.75, device="cuda")          # pads hold non-data
    Pd[:, :S] = torch.from_numpy(P).cuda()
    G = torch.full((N, ld), float("nan"), device="cuda")
    W = (S + 31) // 32
    bits = torch.zeros((N, W), dtype=torch.int32, device="cuda")
    terms = torch.zeros(4 * S + 1, device="cuda")
    scratch = torch.empty(cpra.cpra_op_loss_scratch_bytes(N, S), dtype=torch.uint8, device="cuda")
    rpd, cold = dev_csr(rp, col)
    lamd = torch.from_numpy(lam).cuda()
    cpra.cpra_op_loss(rpd, cold, Pd, lamd, problem, alpha, gamma, nu, div, grad_kind, G, bits,
                      terms, scratch)
    torch.cuda.synchronize()
    Gh = G.cpu().numpy()
    th = terms.cpu().numpy().astype(np.float64)

    ref = O.loss_terms(g, P, lam, problem, alpha, div)
    GP = O.grad_P(g, P, lam, problem, alpha, gamma, nu, div)
    P64 = P.astype(np.float64)
    Gref = GP * P64 * (1 - P64) if grad_kind == 0 else GP
    # pads written as exact zeros
    assert np.all(Gh[:, S:] == 0.0)
    err = np.linalg.norm(Gh[:, :S] - Gref) / np.linalg.norm(Gref)
    assert err <= 1e-5, err
    assert np.abs(Gh[:, :S] - Gref).max() <= 1e-5 * np.abs(Gref).max()
    cost, pen, ann, psi, gsum = th[:S], th[S:2 * S], th[2 * S:3 * S], th[3 * S], th[3 * S + 1:]
    lam64 = lam.astype(np.float64) if problem == O.MIS else np.zeros(S)
    norm = np.abs(ref["cost"]) + lam64 * np.abs(ref["pen"]) + abs(gamma) * ref["ann"]
    Lg = cost + lam64 * pen + gamma * ann
    Lr = ref["cost"] + lam64 * ref["pen"] + gamma * ref["ann"]
    assert np.max(np.abs(Lg - Lr) / norm) <= 1e-5
    assert np.max(np.abs(ann - ref["ann"]) / ref["ann"]) <= 1e-5
    assert abs(psi - ref["psi"]) <= 1e-5 * abs(ref["psi"])
    assert np.max(np.abs(gsum - Gref.sum(axis=0))) <= 1e-5 * np.abs(Gref).sum(axis=0).max()
    # rounding bits are exact
    bh = bits.cpu().numpy().view(np.uint32)
    assert np.array_equal(bh, O.pack_bits(O.round_solutions(P)))


@pytest.mark.parametrize("alpha", [2, 4])
def test_op_loss_annealing_term_near_integral_P(alpha):
    """Late in annealing P sits next to 0 or 1, where 1 - (2P-1)^alpha is a
    difference of nearly equal numbers; the per-shot annealing sums (which
    the early-stopping threshold reads) keep FP32 relative accuracy there."""
    N, S = 20000, 16
    rp, col = I.random_regular_graph(N, 3, seed=8)
    rng = np.random.default_rng(2)
    eps = np.float32(10.0) ** rng.uniform(-6, -3, size=(N, S)).astype(np.float32)
    P = np.where(rng.random((N, S)) < 0.5, eps, np.float32(1) - eps).astype(np.float32)
    ld = rup(S, 16)
    rpd, cold = dev_csr(rp, col)
    Pd = torch.zeros((N, ld), device="cuda")
    Pd[:, :S] = torch.from_numpy(P).cuda()
    G = torch.zeros((N, ld), device="cuda")
    terms = torch.zeros(4 * S + 1, device="cuda")
    scratch = torch.empty(cpra.cpra_op_loss_scratch_bytes(N, S), dtype=torch.uint8, device="cuda")
    lam = torch.ones(S, device="cuda")
    cpra.cpra_op_loss(rpd, cold, Pd, lam, O.MIS, alpha, -1.0, 0.0, O.DIV_STD, 0, G, None, terms,
                      scratch)
    ann = terms.cpu().numpy()[2 * S:3 * S].astype(np.float64)
    ref = O.loss_terms(O.Graph(rp, col), P, np.ones(S), O.MIS, alpha)["ann"]
    assert np.max(np.abs(ann - ref) / ref) <= 1e-5


def test_op_loss_constant_rows_have_zero_diversity_gradient():
    N, S = 64, 16
    rp, col = I.random_regular_graph(N, 3, seed=3)
    P = np.full((N, S), 0.3, dtype=np.float32)
    P[::2] = np.float32(1 / 3)
    ld = rup(S, 16)
    rpd, cold = dev_csr(rp, col)
    Pd = torch.from_numpy(P).cuda()
    G = torch.zeros((N, ld), device="cuda")
    terms = torch.zeros(4 * S + 1, device="cuda")
    scratch = torch.empty(cpra.cpra_op_loss_scratch_bytes(N, S), dtype=torch.uint8, device="cuda")
    lam = torch.ones(S, device="cuda")
    cpra.cpra_op_loss(rpd, cold, Pd, lam, O.MIS, 2, 0.0, 5.0, O.DIV_STD, 1, G, None, terms,
                      scratch)
    g = O.Graph(rp, col)
    Gref = O.grad_P(g, P, np.ones(S), O.MIS, 2, 0.0, 5.0, O.DIV_STD)
    assert np.allclose(G.cpu().numpy(), Gref, rtol=1e-6, atol=1e-6)
    assert terms[3 * S].item() == 0.0


# =============================================================== round/eval
@pytest.mark.parametrize("problem", [O.MIS, O.MAXCUT])
# The S values reach every layout of the evaluation kernel: one 32-shot word
# per lane for odd word counts (S = 1, 8: 8 lanes a row; 270: 16; 530: 32)
# and two words per lane for even counts (37, 100: 2 lanes; 256: 4; 300: 8;
# 640, 1000: 16), with rows long enough for several neighbour passes and
# slot groups (degrees 20-40).
@pytest.mark.parametrize("S,N,gk", [(8, 1000, ("rrg", 3)), (37, 2001, ("er", 6)),
                                     (100, 1500, ("rrg", 20)), (256, 999, ("er", 5)),
                                     (1000, 200, ("er", 3)), (1, 50, ("rrg", 4)),
                                     (300, 700, ("rrg", 9)), (270, 500, ("er", 12)),
                                     (530, 300, ("er", 40)), (640, 400, ("er", 30))])
def test_op_round_eval_bit_exact(problem, S, N, gk):
    rp, col = graph_of(gk, N, seed=7 * S + N)
    g = O.Graph(rp, col)
    P = I.seeded_P(N, S, seed=S)
    lam = I.lambda_linspace(1.0, 8.0, S)
    ld = rup(S, 4)
    Pd = torch.full((N, ld), 0.9, device="cuda")
    Pd[:, :S] = torch.from_numpy(P).cuda()
    W = (S + 31) // 32
    bits = torch.zeros((N, W), dtype=torch.int32, device="cuda")
    rec = torch.zeros(S * 4, dtype=torch.float64, device="cuda")  # cpra_shot_eval [S]
    ham = torch.zeros(1, dtype=torch.int64, device="cuda")
    cnt = torch.empty(cpra.cpra_op_round_eval_scratch_bytes(S), dtype=torch.uint8, device="cuda")
    rpd, cold = dev_csr(rp, col)
    cpra.cpra_op_round_eval(rpd, cold, Pd, S, torch.from_numpy(lam).cuda(), problem, bits, rec,
                            ham, cnt)
    torch.cuda.synchronize()
    r = rec.cpu().numpy().view(cpra.SHOT_EVAL_DTYPE)
    Xr = O.round_solutions(P)
    ev = O.integer_eval(g, Xr, lam.astype(np.float64), problem)
    assert np.array_equal(r["objective"], ev["objective"])
    assert np.array_equal(r["violations"], ev["violations"])
    assert np.array_equal(r["qubo"], ev["qubo"])
    assert int(ham.item()) == ev["pair_hamming"]
    assert np.array_equal(bits.cpu().numpy().view(np.uint32), O.pack_bits(Xr))


def test_op_round_eval_threshold_edge_cases():
    """P exactly 0.5 rounds to 0; P all above 0.5 selects every node."""
    N, S = 300, 40
    rp, col = I.random_regular_graph(N, 4, seed=1)
    rpd, cold = dev_csr(rp, col)
    lam = torch.full((S,), 2.0, device="cuda")
    for val, sel in ((0.5, 0), (np.nextafter(np.float32(0.5), np.float32(1)), 1)):
        Pd = torch.full((N, S), float(val), device="cuda")
        bits = torch.zeros((N, 2), dtype=torch.int32, device="cuda")
        rec = torch.zeros(S * 4, dtype=torch.float64, device="cuda")  # cpra_shot_eval [S]
        ham = torch.zeros(1, dtype=torch.int64, device="cuda")
        cnt = torch.empty(cpra.cpra_op_round_eval_scratch_bytes(S), dtype=torch.uint8, device="cuda")
        cpra.cpra_op_round_eval(rpd, cold, Pd, S, lam, O.MIS, bits, rec, ham, cnt)
        r = rec.cpu().numpy().view(cpra.SHOT_EVAL_DTYPE)
        assert np.all(r["objective"] == sel * N)
        assert np.all(r["violations"] == sel * (len(col) // 2))
        assert ham.item() == 0


# ================================================================ full step
def oracle_cfg(S, H0, H1, problem, alpha, lam, gamma, nu, div, train_emb=True):
    return dict(H0=H0, H1=H1, S=S, problem=problem, alpha=alpha,
                lam=np.asarray(lam, np.float64), gamma=gamma, nu=nu, div_kind=div, lr=1e-3,
                beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0, train_embedding=train_emb)


STEP_CASES = [
    # problem, div, alpha, nu, S, H, N, graph
    (O.MIS, O.DIV_STD, 2, 0.0, 8, 16, 100, ("rrg", 3)),
    (O.MIS, O.DIV_STD, 4, 0.3, 24, 32, 700, ("er", 5)),
    (O.MAXCUT, O.DIV_VAR, 2, 0.1, 64, 32, 1200, ("er", 10)),
    (O.MAXCUT, O.DIV_STD, 2, 0.2, 100, 48, 517, ("rrg", 20)),
    # H = 256: the layer-1 weights (256 x 512 BF16) exceed shared memory as one
    # tile, so the tensor-core GEMM splits the output columns into two tiles
    (O.MIS, O.DIV_STD, 2, 0.0, 100, 256, 600, ("rrg", 20)),
    # H = 1040 (wide layers): the aggregations run as two column slices, the
    # dense layers stream their weights with the A stages and end in a
    # ragged n tile (1040 = 4 x 256 + 16)
    (O.MAXCUT, O.DIV_STD, 2, 0.2, 40, 1040, 700, ("rrg", 4)),
]


def _run_step_case(case, precision, keep_emb_grad=1, recompute=0, init_logits=None, plain=False,
                   fp32_engine=0, weights=None):
    """One GPU step from seeded state and the oracle's step from the same
    state.  With plain=True the BF16 form is also compared with the oracle
    that decides the ReLU signs on FP64 Z1 (out["ref_plain"]).  ``weights``
    ("uniform" or "pm1") gives a MaxCut case seeded edge weights A_ij."""
    problem, div, alpha, nu, S, H, N, gk = case
    rp, col = graph_of(gk, N, seed=N + S)
    w = None if weights is None else I.seeded_edge_weights(rp, col, seed=S, kind=weights)
    g = O.Graph(rp, col, weights=w)
    lam = I.lambda_geomspace(0.5, 10.0, S)
    theta, X0 = I.seeded_params(N, H, H, S, seed=5, weight_scale=1.5)
    mt, vt = I.seeded_adam_state(len(theta), seed=6)
    mx, vx = I.seeded_adam_state(N * H, seed=7)
    t_prev, t_idx, T = 5, 3, 11
    gamma = O.gamma_schedule(t_idx, T, -1.0, 1.0)
    solver = cpra.Solver(rp, col, lam=lam if problem == O.MIS else None, problem=problem, S=S,
                         H0=H, H1=H, alpha=alpha, precision=precision, nu=nu,
                         diversity_kind=div, gamma0=-1.0, gamma1=1.0, schedule_steps=T,
                         keep_emb_grad=keep_emb_grad, recompute=recompute, fp32_engine=fp32_engine,
                         weights=w)
    for which, arr in ((cpra.T_THETA, theta), (cpra.T_EMB, X0), (cpra.T_THETA_M, mt),
                       (cpra.T_THETA_V, vt), (cpra.T_EMB_M, mx), (cpra.T_EMB_V, vx),
                       (cpra.T_STEP, np.array([t_prev]))):
        solver.set(which, arr)
    if init_logits is not None:
        solver.set_init_logits(init_logits)
    terms = solver.step(t_idx, want_terms=True).astype(np.float64)
    out = dict(P=solver.P(), grad=solver.get(cpra.T_GRAD), gX0=solver.get(cpra.T_EMB_GRAD),
               theta=solver.get(cpra.T_THETA), X0=solver.get(cpra.T_EMB), terms=terms,
               X0_m=solver.get(cpra.T_EMB_M), X0_v=solver.get(cpra.T_EMB_V))
    rec, ham, bits = solver.round_eval(want_bits=True)
    out.update(rec=rec, ham=ham, bits=bits, adam0=(mt, vt, mx, vx, t_prev + 1))
    assert solver.get(cpra.T_STEP)[0] == t_prev + 1
    solver.close()
    cfg = oracle_cfg(S, H, H, problem, alpha, lam, gamma, nu, div)
    if precision == cpra.BF16:
        # the ReLU sign is decided at the kernels' (bfloat16 operand) precision
        cfg["relu_decision"] = "bf16"
    if init_logits is not None:
        # the library keeps the offset in the dense layers' dtype
        cfg["init_logits"] = (O.bf16_round(init_logits) if precision == cpra.BF16
                              else np.asarray(init_logits, dtype=np.float64))
    adam_state = dict(m_theta=mt, v_theta=vt, m_X0=mx.reshape(N, H), v_X0=vx.reshape(N, H))
    ref = O.step(g, theta, X0, cfg, t=t_prev + 1, adam_state=adam_state)
    if plain:
        cfg_plain = dict(cfg)
        cfg_plain.pop("relu_decision", None)
        out["ref_plain"] = O.step(g, theta, X0, cfg_plain, t=t_prev + 1, adam_state=adam_state)
    return out, ref, g, lam, gamma, theta, X0


def _step_errors(out, ref, lam, gamma, S, H, problem):
    """The parity measures of one step against one oracle result: max |dP|,
    the per-shot loss error over the cancellation-safe normaliser, Psi
    relative to |Psi|, and the norm-wise relative error of each parameter
    gradient block and of the embedding gradient."""
    e = {"P": float(np.abs(out["P"] - ref["P"]).max())}
    t = out["terms"]
    lam64 = lam.astype(np.float64) if problem == O.MIS else np.zeros(S)
    rt = ref["terms"]
    norm = np.abs(rt["cost"]) + lam64 * np.abs(rt["pen"]) + abs(gamma) * rt["ann"]
    Lg = t[:S] + lam64 * t[S:2 * S] + gamma * t[2 * S:3 * S]
    Lr = rt["cost"] + lam64 * rt["pen"] + gamma * rt["ann"]
    e["loss"] = float(np.max(np.abs(Lg - Lr) / norm))
    e["psi"] = float(abs(t[3 * S] - rt["psi"]) / abs(rt["psi"])) if rt["psi"] != 0 else 0.0
    lay = I.param_layout(H, H, S)
    for name in ("Wcat1", "b1", "Wcat2", "b2"):
        off, shape = lay[name]
        n = int(np.prod(shape))
        a, b = out["grad"][off:off + n], ref["grads"]["theta"][off:off + n]
        e[name] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    gX = ref["grads"]["X0"]
    e["X0"] = float(np.linalg.norm(out["gX0"].reshape(gX.shape) - gX) / np.linalg.norm(gX))
    return e


def _check_step(out, ref, g, lam, gamma, theta, X0, S, H, tol, problem):
    e = _step_errors(out, ref, lam, gamma, S, H, problem)
    for k, v in e.items():
        assert v <= tol, (k, v)
    # Adam: the step taken equals Adam (FP64) applied to the step's own
    # gradients, which the checks above hold to the oracle's
    mt, vt, mx, vx, tt = out["adam0"]
    th_exp = O.adam(theta, mt, vt, out["grad"], tt, lr=1e-3)[0]
    assert np.linalg.norm(out["theta"] - th_exp) <= 1e-4 * np.linalg.norm(th_exp - theta)
    x_exp = O.adam(X0.reshape(-1), mx, vx, out["gX0"], tt, lr=1e-3)[0].reshape(X0.shape)
    assert np.linalg.norm(out["X0"].reshape(X0.shape) - x_exp) <= 1e-4 * np.linalg.norm(x_exp - X0)
    # and the oracle's own step, for the smaller layers: with millions of
    # parameters some seeded second moments are tiny, where Adam's update is
    # sign-like and turns gradient rounding into full-size differences
    if len(theta) < 10**6:
        dref = ref["theta_next"] - theta
        assert np.linalg.norm(out["theta"] - ref["theta_next"]) <= 10 * tol * np.linalg.norm(dref)
        dref = ref["X0_next"] - X0
        assert np.linalg.norm(out["X0"].reshape(X0.shape) - ref["X0_next"]) <= 10 * tol * np.linalg.norm(dref)


@pytest.mark.parametrize("engine", [cpra.FP32_TENSOR, cpra.FP32_CUDA_CORES])
@pytest.mark.parametrize("case", STEP_CASES)
def test_full_step_fp32_matches_oracle(case, engine):
    """Both engines of the FP32 form: split-TF32 tensor-core GEMMs (the
    default) and CUDA-core GEMMs, each within 1e-5 of the FP64 oracle."""
    out, ref, g, lam, gamma, theta, X0 = _run_step_case(case, cpra.FP32, fp32_engine=engine)
    problem, S, H = case[0], case[4], case[5]
    _check_step(out, ref, g, lam, gamma, theta, X0, S, H, 1e-5, problem)
    # rounding: bit-exact wherever the FP64 P is not within tolerance of 0.5
    x_gpu = unpack_bits(out["bits"], S)
    decided = np.abs(ref["P"] - 0.5) > 1e-5
    assert np.array_equal(x_gpu[decided], ref["X"][decided])
    if decided.all():
        ev = ref["eval"]
        assert np.array_equal(out["rec"]["objective"], ev["objective"])
        assert np.array_equal(out["rec"]["violations"], ev["violations"])
        assert out["ham"] == ev["pair_hamming"]


# Quantities that the layer-1 ReLU decisions cannot move by more than the
# rounding of the values they gate: H1 = max(Z1, 0) is continuous where a
# sign flips, so P, the loss terms and the layer-2 gradients (dWcat2 =
# G_Z2^T [H1 | M2]) stay close to FP64 whichever precision decides the sign.
# The layer-1 and embedding gradients carry G_Z1 = G_H1 * 1[Z1 > 0], which a
# flipped sign changes by a whole G_H1 entry.
MASK_CONTINUOUS = ("P", "loss", "psi", "Wcat2", "b2")


def _report_plain(name, case, e_matched, e_plain):
    """Appends one JSON line per case to $CPRA_PARITY_REPORT (if set): the
    BF16 form's parity measures against the decision-matched and the plain
    FP64 oracle."""
    import json
    import os
    path = os.environ.get("CPRA_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": name, "case": [str(c) for c in case],
                                "vs_matched_fp64": e_matched, "vs_plain_fp64": e_plain}) + "\n")


@pytest.mark.parametrize("case", STEP_CASES)
def test_full_step_bf16_matches_oracle(case):
    out, ref, g, lam, gamma, theta, X0 = _run_step_case(case, cpra.BF16, plain=True)
    _check_step(out, ref, g, lam, gamma, theta, X0, case[4], case[5], 2e-2, case[0])
    # against the plain FP64 oracle (every ReLU sign decided on FP64 Z1): the
    # mask-continuous results meet the same 2e-2 bar; the layer-1 gradients
    # are reported
    e_m = _step_errors(out, ref, lam, gamma, case[4], case[5], case[0])
    e_p = _step_errors(out, out["ref_plain"], lam, gamma, case[4], case[5], case[0])
    _report_plain("full_step_bf16", case, e_m, e_p)
    for k in MASK_CONTINUOUS:
        assert e_p[k] <= 2e-2, (k, e_p[k])


@pytest.mark.parametrize("precision", [cpra.FP32, cpra.BF16])
def test_fused_embedding_update_without_stored_gradient(precision):
    """By default the step fuses the embedding Adam update into the last
    backward aggregation and does not store dR/dh^0; the updated embeddings
    and moments are bit-identical to the run that also stores the gradient,
    and both match the oracle's Adam step (Experiments section optimiser)."""
    case = STEP_CASES[0]
    S, H = case[4], case[5]
    kept, ref, g, lam, gamma, theta, X0 = _run_step_case(case, precision, keep_emb_grad=1)
    fused, _, _, _, _, _, _ = _run_step_case(case, precision, keep_emb_grad=0)
    for k in ("X0", "X0_m", "X0_v", "theta", "grad", "P"):
        assert np.array_equal(kept[k], fused[k]), k
    tol = 1e-5 if precision == cpra.FP32 else 2e-2
    dref = ref["X0_next"] - X0
    assert np.linalg.norm(fused["X0"].reshape(X0.shape) - ref["X0_next"]) <= 10 * tol * np.linalg.norm(dref)


@pytest.mark.parametrize("precision", [cpra.FP32, cpra.BF16])
@pytest.mark.parametrize("ci", [0, 2])
def test_full_step_with_init_logits_matches_oracle(precision, ci):
    """Warm-start offset L0 on the head's pre-activation (cpra_set_init_logits)
    through a full step, against the oracle forward with the same offset."""
    case = STEP_CASES[ci]
    S, N = case[4], case[6]
    L0 = np.random.default_rng(11).normal(size=(N, S)).astype(np.float32) * 2.0
    tol = 1e-5 if precision == cpra.FP32 else 2e-2
    out, ref, g, lam, gamma, theta, X0 = _run_step_case(case, precision, init_logits=L0)
    _check_step(out, ref, g, lam, gamma, theta, X0, S, case[5], tol, case[0])


def test_init_logits_cleared_restores_plain_network():
    rp, col = I.random_regular_graph(200, 3, seed=5)
    lam = I.lambda_linspace(1, 4, 8)
    a = cpra.Solver(rp, col, lam=lam, problem=cpra.MIS, S=8, seed=2)
    b = cpra.Solver(rp, col, lam=lam, problem=cpra.MIS, S=8, seed=2)
    b.set_init_logits(np.full((200, 8), 3.0, np.float32))
    b.set_init_logits(None)
    for t in range(3):
        a.step(t)
        b.step(t)
    assert np.array_equal(a.P(), b.P())
    # ld < S is rejected
    st = cpra.lib().cpra_set_init_logits(a.ctx, cpra._ptr(np.zeros(8, np.float32)), 4, 0)
    assert st == cpra.CPRA_EINVAL
    a.close()
    b.close()


@pytest.mark.parametrize("ci", [1, 5])
@pytest.mark.parametrize("precision", [cpra.FP32, cpra.BF16])
def test_recompute_step_matches_oracle_and_stored_form(precision, ci):
    """recompute = 1 (the layer-1 adjoint's ReLU mask recomputed from Z1, the
    activation blocks shared with the gradient blocks) gives the same step
    bit for bit as the stored-activation form, and matches the oracle."""
    case = STEP_CASES[ci]
    S, H = case[4], case[5]
    tol = 1e-5 if precision == cpra.FP32 else 2e-2
    stored, ref, g, lam, gamma, theta, X0 = _run_step_case(case, precision, recompute=0)
    lean, _, _, _, _, _, _ = _run_step_case(case, precision, recompute=1)
    for k in ("P", "grad", "gX0", "theta", "X0", "X0_m", "X0_v", "terms", "bits"):
        assert np.array_equal(stored[k], lean[k]), k
    _check_step(lean, ref, g, lam, gamma, theta, X0, S, H, tol, case[0])


@pytest.mark.parametrize("precision", [cpra.FP32, cpra.BF16])
def test_recompute_many_steps_bitwise(precision):
    """Five steps with and without recompute from the same seed stay
    bit-identical (P, parameters, embeddings and the rounded bits)."""
    rp, col = I.random_regular_graph(3000, 5, seed=21)
    lam = I.lambda_linspace(1, 8, 48)
    outs = []
    for rc in (0, 1):
        s = cpra.Solver(rp, col, lam=lam, problem=cpra.MIS, S=48, H0=32, H1=48,
                        precision=precision, nu=0.2, seed=7, recompute=rc)
        for t in range(5):
            s.step(t)
        rec, ham, bits = s.round_eval(want_bits=True)
        outs.append((s.P(), s.get(cpra.T_THETA), s.get(cpra.T_EMB), bits, rec["objective"]))
        s.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [cpra.FP32, cpra.BF16])
def test_eval_records_match_returned_bits(precision):
    """The per-shot records of a step are exactly the objective of the bits
    the same call returns (validity of the fused evaluation)."""
    N, S = 400, 40
    rp, col = I.random_regular_graph(N, 3, seed=9)
    adj = X.adjacency_sets(rp, col)
    lam = I.lambda_linspace(1, 8, S)
    solver = cpra.Solver(rp, col, lam=lam, problem=cpra.MIS, S=S, H0=16, H1=16,
                         precision=precision, schedule_steps=50)
    for t in range(30):
        solver.step(t)
    rec, ham, bits = solver.round_eval(want_bits=True)
    x = unpack_bits(bits, S)
    for s in range(S):
        inside = sum(1 for i in range(N) for j in adj[i] if i < j and x[i, s] and x[j, s])
        assert rec["objective"][s] == x[:, s].sum()
        assert rec["violations"][s] == inside
        assert rec["qubo"][s] == -float(x[:, s].sum()) + float(lam[s]) * inside
    k = x.sum(axis=1)
    assert ham == int((k * (S - k)).sum())
    solver.close()


# ================================================= checkpoint / determinism
@pytest.mark.parametrize("precision", [cpra.FP32, cpra.BF16])
def test_resume_is_bitwise_identical(precision):
    N, S = 2000, 32
    rp, col = I.random_regular_graph(N, 5, seed=4)
    lam = I.lambda_geomspace(0.5, 10, S)
    kw = dict(lam=lam, problem=cpra.MIS, S=S, H0=32, H1=32, precision=precision, nu=0.2,
              schedule_steps=20, seed=3)
    a = cpra.Solver(rp, col, **kw)
    for t in range(3):
        a.step(t)
    blob = cpra.cpra_get_state(a.ctx)
    for t in range(3, 6):
        a.step(t)
    th_a, x_a = a.get(cpra.T_THETA), a.get(cpra.T_EMB)
    b = cpra.Solver(rp, col, **dict(kw, seed=99))
    cpra.cpra_set_state(b.ctx, blob)
    for t in range(3, 6):
        b.step(t)
    assert np.array_equal(th_a, b.get(cpra.T_THETA))
    assert np.array_equal(x_a, b.get(cpra.T_EMB))
    a.close()
    b.close()


def test_state_mismatch_is_rejected():
    rp, col = I.random_regular_graph(100, 3, seed=1)
    a = cpra.Solver(rp, col, lam=np.ones(8, np.float32), problem=cpra.MIS, S=8)
    blob = cpra.cpra_get_state(a.ctx)
    b = cpra.Solver(rp, col, lam=np.ones(16, np.float32), problem=cpra.MIS, S=16)
    with pytest.raises(cpra.CpraError) as ei:
        cpra.cpra_set_state(b.ctx, blob)
    assert ei.value.status == cpra.CPRA_ESTATE
    a.close()
    b.close()


def test_non_finite_loss_is_reported():
    """Fault injection on the host: NaN parameters make the step report
    CPRA_ENUMERIC instead of silently continuing."""
    rp, col = I.random_regular_graph(100, 3, seed=1)
    s = cpra.Solver(rp, col, lam=np.ones(8, np.float32), problem=cpra.MIS, S=8)
    th = s.get(cpra.T_THETA)
    th[-1] = np.nan
    s.set(cpra.T_THETA, th)
    with pytest.raises(cpra.CpraError) as ei:
        s.step(0, want_terms=True)
    assert ei.value.status == cpra.CPRA_ENUMERIC
    s.close()


def test_profiling_and_launch_counts():
    rp, col = I.random_regular_graph(1000, 3, seed=1)
    s = cpra.Solver(rp, col, lam=np.ones(8, np.float32), problem=cpra.MIS, S=8)
    cpra.cpra_profile_enable(s.ctx, True)
    n0 = s.launches
    for t in range(4):
        s.step(t)
    prof = cpra.cpra_profile_read(s.ctx)
    assert prof["loss_fused"][1] == 4 and prof["loss_fused"][0] > 0
    assert s.launches - n0 >= 4 * 12
    s.close()


# ================================================================ behaviour
def test_small_rrg_reaches_exact_mis():
    """Variation-diversified MIS on seeded 30-node 3-regular graphs (the
    shape of the paper's small instance): the best feasible shot reaches the
    exact independence number from branch and bound."""
    hits = 0
    for seed in (1, 2, 3):
        rp, col = I.random_regular_graph(30, 3, seed=seed)
        alpha_g = X.max_independent_set_size(X.adjacency_sets(rp, col))
        S = 100
        s = cpra.Solver(rp, col, lam=np.full(S, 2.0, np.float32), problem=cpra.MIS, S=S,
                        H0=16, H1=16, nu=0.5, gamma0=-2.0, gamma1=0.1, schedule_steps=3000,
                        seed=seed)
        best, _ = s.solve(3000, 100)
        feas = best["objective"]
        assert feas.max() <= alpha_g
        hits += int(feas.max() == alpha_g)
        s.close()
    assert hits >= 2
