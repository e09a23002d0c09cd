"""The relaxed loss as a torch.autograd.Function whose backward is the
library's hand-written adjoint: checked against the FP64 oracle gradient and
against central finite differences of the same forward."""
import numpy as np
import pytest

from oracle import cpra_oracle as O
from paper_2402_02190_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2402_02190_gb300 import cpra  # noqa: E402
from paper_2402_02190_gb300.autograd import cpra_loss  # noqa: E402


def _setup(precision, problem=cpra.MIS, nu=0.3, div=cpra.DIV_STD, N=600, S=40, H=32, seed=3):
    rp, col = I.random_regular_graph(N, 4, seed)
    lam = I.lambda_geomspace(0.5, 10.0, S)
    solver = cpra.Solver(rp, col, lam=lam if problem == cpra.MIS else None, problem=problem, S=S,
                         H0=H, H1=H, precision=precision, nu=nu, diversity_kind=div)
    theta, X0 = I.seeded_params(N, H, H, S, seed=seed + 10, weight_scale=1.5)
    return solver, rp, col, lam, theta, X0


@pytest.mark.parametrize("precision,tol", [(cpra.FP32, 1e-5), (cpra.BF16, 2e-2)])
@pytest.mark.parametrize("problem,div", [(cpra.MIS, cpra.DIV_STD), (cpra.MAXCUT, cpra.DIV_VAR)])
def test_autograd_gradient_matches_oracle(precision, tol, problem, div):
    solver, rp, col, lam, theta, X0 = _setup(precision, problem, div=div)
    N, S, H = solver.N, solver.S, 32
    gamma = -0.45
    th = torch.tensor(theta, device="cuda", requires_grad=True)
    em = torch.tensor(X0, device="cuda", requires_grad=True)
    R, terms = cpra_loss(solver, th, em, gamma)
    R.backward()
    g = O.Graph(rp, col)
    lam64 = lam.astype(np.float64) if problem == cpra.MIS else np.zeros(S)
    c = O.forward(g, theta, X0, H, H, S, relu_decision="bf16" if precision == cpra.BF16 else None)
    t = O.loss_terms(g, c["P"], lam64, problem, 2, div)
    R_ref = O.total_loss(t, lam64, gamma, 0.3, problem)
    GP = O.grad_P(g, c["P"], lam64, problem, 2, gamma, 0.3, div)
    gr = O.backward(g, theta, c, GP, H, H, S)
    norm = (np.abs(t["cost"]).sum() + (lam64 * np.abs(t["pen"])).sum() + abs(gamma) * t["ann"].sum()
            + 0.3 * abs(t["psi"]))
    assert abs(R.item() - R_ref) <= tol * norm
    lay = I.param_layout(H, H, S)
    gt = th.grad.cpu().numpy().astype(np.float64)
    for name in ("Wcat1", "b1", "Wcat2", "b2"):
        off, shape = lay[name]
        n = int(np.prod(shape))
        e = np.linalg.norm(gt[off:off + n] - gr["theta"][off:off + n]) / np.linalg.norm(gr["theta"][off:off + n])
        assert e <= tol, (name, e)
    ge = em.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(ge - gr["X0"]) <= tol * np.linalg.norm(gr["X0"])
    solver.close()


@pytest.mark.parametrize("precision", [cpra.FP32, cpra.BF16])
def test_autograd_recompute_matches_stored(precision):
    """With recompute = 1 the adjoint (whose gradient block overwrites the
    embedding copy the forward reads) gives the same gradients, and the next
    forward sees the restored copy: two forward/backward rounds are
    bit-identical to the stored-activation form."""
    res = []
    for rc in (0, 1):
        rp, col = I.random_regular_graph(600, 4, 3)
        lam = I.lambda_geomspace(0.5, 10.0, 40)
        solver = cpra.Solver(rp, col, lam=lam, problem=cpra.MIS, S=40, H0=32, H1=32,
                             precision=precision, nu=0.3, recompute=rc)
        theta, X0 = I.seeded_params(600, 32, 32, 40, seed=13, weight_scale=1.5)
        out = []
        for _ in range(2):
            th = torch.tensor(theta, device="cuda", requires_grad=True)
            em = torch.tensor(X0, device="cuda", requires_grad=True)
            R, _ = cpra_loss(solver, th, em, -0.3)
            R.backward()
            out += [R.item(), th.grad.cpu().numpy(), em.grad.cpu().numpy()]
        # a training step after the autograd backward reads the restored copy
        solver.step(0)
        out.append(solver.P())
        res.append(out)
        solver.close()
    for a, b in zip(*res):
        assert np.array_equal(np.asarray(a), np.asarray(b))


def test_autograd_directional_finite_differences():
    """(R(p + h v) - R(p - h v)) / 2h against grad . v, for random directions
    v over (theta, h^0), all through the library's FP32 forward."""
    solver, rp, col, lam, theta, X0 = _setup(cpra.FP32, N=400, S=24, H=16)
    gamma = 0.2
    th = torch.tensor(theta, device="cuda", requires_grad=True)
    em = torch.tensor(X0, device="cuda", requires_grad=True)
    R, _ = cpra_loss(solver, th, em, gamma)
    R.backward()
    gt, ge = th.grad.double(), em.grad.double()
    gnorm = torch.sqrt((gt ** 2).sum() + (ge ** 2).sum()).item()
    gen = torch.Generator(device="cuda").manual_seed(0)
    for k in range(4):
        vt = torch.randn(th.shape, generator=gen, device="cuda", dtype=torch.float64)
        ve = torch.randn(em.shape, generator=gen, device="cuda", dtype=torch.float64)
        nv = torch.sqrt((vt ** 2).sum() + (ve ** 2).sum())
        vt, ve = vt / nv, ve / nv
        h = 1.0 / gnorm * 0.5
        with torch.no_grad():
            Rp, _ = cpra_loss(solver, (th.double() + h * vt).float(), (em.double() + h * ve).float(), gamma)
            Rm, _ = cpra_loss(solver, (th.double() - h * vt).float(), (em.double() - h * ve).float(), gamma)
        fd = (Rp.double() - Rm.double()).item() / (2 * h)
        an = ((gt * vt).sum() + (ge * ve).sum()).item()
        assert abs(fd - an) <= 2e-2 * gnorm, (k, fd, an, gnorm)
    solver.close()


def test_autograd_adam_step_matches_cpra_step():
    """One torch.optim.Adam step on the autograd gradient equals the
    library's own fused step (FP32 form, same state)."""
    solver, rp, col, lam, theta, X0 = _setup(cpra.FP32, N=500, S=16, H=16, nu=0.0)
    T = 5
    gamma = -2.0
    th = torch.tensor(theta, device="cuda", requires_grad=True)
    em = torch.tensor(X0, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([th, em], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    R, _ = cpra_loss(solver, th, em, gamma)
    R.backward()
    opt.step()
    ref = cpra.Solver(rp, col, lam=lam, problem=cpra.MIS, S=16, H0=16, H1=16,
                      precision=cpra.FP32, nu=0.0, gamma0=gamma, gamma1=gamma, schedule_steps=T)
    ref.set(cpra.T_THETA, theta)
    ref.set(cpra.T_EMB, X0)
    ref.step(0)
    d_ref = ref.get(cpra.T_THETA) - theta
    d_got = th.detach().cpu().numpy() - theta
    assert np.linalg.norm(d_got - d_ref) <= 1e-3 * np.linalg.norm(d_ref)
    e_ref = ref.get(cpra.T_EMB).reshape(X0.shape) - X0
    e_got = em.detach().cpu().numpy() - X0
    assert np.linalg.norm(e_got - e_ref) <= 1e-3 * np.linalg.norm(e_ref)
    ref.close()
    solver.close()


def test_backward_without_forward_is_a_state_error():
    solver, *_ = _setup(cpra.FP32, N=100, S=8, H=16)
    g = torch.empty(cpra.cpra_param_count(solver.ctx), device="cuda")
    with pytest.raises(cpra.CpraError) as ei:
        cpra.cpra_backward(solver.ctx, 1.0, g)
    assert ei.value.status == cpra.CPRA_ESTATE
    solver.close()
