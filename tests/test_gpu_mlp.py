"""GPU kernels of the learned preconditioner against the CPU oracle (oracle/mlp.py):
potential diagonal, loss and gradients (BF16 weights, FP32 arithmetic vs FP64 reference),
inference equal to TPA for a zero last layer, training lowers the loss, traced solves."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import basis as B
from oracle import mlp as Mo
from oracle import potential as P
from paper_2210_12252_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hwmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_12252_gb300 import build
    build.build()
    from paper_2210_12252_gb300 import helicwave
    return helicwave


@pytest.fixture(scope="module")
def case(hwmod):
    w = inputs.tiny()
    g = w.geom
    eta, ecut = 0.1, 12.0
    ctx = hwmod.Context(0)
    ctx.setup_basis(g, [eta], None, [ecut])
    ctx.build_potential(w.atoms)
    params = Mo.init_params(3)
    params[4] = np.random.default_rng(8).standard_normal(Mo.HIDDEN) * 0.2
    params[5] = np.array([0.1])
    flat = np.concatenate([p.reshape(-1) for p in params]).astype(np.float32)
    ctx.set_mlp(flat)
    b = B.Basis(g.R, g.tau, g.alpha, g.Nr, g.Nth1, g.Nth2)
    kp = B.KPoint(b, eta, 0.0, ecut)
    V = P.gaussian_wells(b, w.atoms)
    return ctx, kp, V, flat


def unflatten(flat):
    f = Mo.bf16_round(np.asarray(flat, dtype=np.float64))
    W1 = f[0:384].reshape(64, 6)
    b1 = f[384:448]
    W2 = f[448:4544].reshape(64, 64)
    b2 = f[4544:4608]
    w3 = f[4608:4672]
    b3 = f[4672:4673]
    return [W1, b1, W2, b2, w3, b3]


def test_potential_diagonal_matches_oracle(case):
    ctx, kp, V, _ = case
    np.testing.assert_allclose(ctx.potential_diagonal(0), Mo.potential_diagonal(kp, V), rtol=1e-12, atol=1e-12)


def test_loss_and_gradient_match_oracle(case):
    ctx, kp, V, flat = case
    rng = np.random.default_rng(5)
    ns = 5
    R = rng.standard_normal((kp.L, ns)) + 1j * rng.standard_normal((kp.L, ns))
    Et = rng.standard_normal((kp.L, ns)) + 1j * rng.standard_normal((kp.L, ns))
    ritz = rng.uniform(-3, 2, ns)
    loss, grad = ctx.mlp_loss_grad(0, torch.from_numpy(np.ascontiguousarray(R.T)).cuda(),
                                   torch.from_numpy(np.ascontiguousarray(Et.T)).cuda(), ritz)
    params = unflatten(flat)
    vd = Mo.potential_diagonal(kp, V)
    ref_loss = 0.0
    ref_grad = [np.zeros_like(p) for p in params]
    for j in range(ns):
        X = Mo.features(kp, vd, ritz[j])
        l, g = Mo.column_loss_and_grad(params, X, Mo.tpa_factor(kp.ke, R[:, j]), R[:, j], Et[:, j])
        ref_loss += l / ns
        for a, b in zip(ref_grad, g):
            a += np.asarray(b) / ns
    gref = np.concatenate([g.reshape(-1) for g in ref_grad])
    assert abs(loss - ref_loss) < 1e-5
    assert np.linalg.norm(grad - gref) < 2e-3 * np.linalg.norm(gref)


def test_zero_last_layer_inference_equals_tpa(hwmod, case):
    """With a zero last layer the network is the TPA diagonal; inference runs in FP32, so the
    two agree to FP32 rounding (a few units of 2^-24 relative per entry)."""
    ctx, kp, V, flat = case
    f0 = flat.copy()
    f0[4608:] = 0.0
    ctx.set_mlp(f0)
    rng = np.random.default_rng(2)
    R = torch.from_numpy(np.ascontiguousarray((rng.standard_normal((kp.L, 4)) + 0j).T)).cuda()
    ritz = torch.tensor([-1.0, 0.0, 0.5, 2.0], dtype=torch.float64, device="cuda")
    Zl = ctx.apply_precond(0, R, ritz=ritz, kind="learned")
    Zt = ctx.apply_precond(0, R, kind="tpa")
    assert ((Zl - Zt).abs() <= 1e-6 * Zt.abs() + 1e-30).all()
    ctx.set_mlp(flat)


def test_inference_matches_oracle_network(hwmod, case):
    """FP32 inference against the oracle's FP64 network on the same BF16 weights: s_i r_i per
    entry to 1e-5 relative (FP32 network arithmetic)."""
    ctx, kp, V, flat = case
    rng = np.random.default_rng(4)
    ns = 3
    R = rng.standard_normal((kp.L, ns)) + 1j * rng.standard_normal((kp.L, ns))
    ritz = np.array([-1.5, 0.2, 1.0])
    Z = ctx.apply_precond(0, torch.from_numpy(np.ascontiguousarray(R.T)).cuda(),
                          ritz=torch.from_numpy(ritz).cuda(), kind="learned").cpu().numpy().T
    params = unflatten(flat)
    vd = Mo.potential_diagonal(kp, V)
    for j in range(ns):
        X = Mo.features(kp, vd, ritz[j])
        s = Mo.tpa_factor(kp.ke, R[:, j]) * np.exp(Mo.forward(params, X)[0])
        np.testing.assert_allclose(Z[:, j], s * R[:, j], rtol=1e-5)


def test_training_steps_lower_the_loss(case):
    ctx, kp, V, flat = case
    rng = np.random.default_rng(11)
    ns = 6
    # target corrections correlated with a mode-dependent rescaling of the residual
    R = rng.standard_normal((kp.L, ns)) + 1j * rng.standard_normal((kp.L, ns))
    Et = R / (1.0 + kp.ke[:, None] + 0.3 * kp.m[:, None] ** 2)
    Rd = torch.from_numpy(np.ascontiguousarray(R.T)).cuda()
    Ed = torch.from_numpy(np.ascontiguousarray(Et.T)).cuda()
    ritz = rng.uniform(-2, 1, ns)
    l0, _ = ctx.mlp_loss_grad(0, Rd, Ed, ritz, want_grad=False)
    for _ in range(60):
        ctx.mlp_train_step(0, Rd, Ed, ritz, 3e-3)
    l1, _ = ctx.mlp_loss_grad(0, Rd, Ed, ritz, want_grad=False)
    assert l1 < 0.5 * l0, (l0, l1)
    ctx.set_mlp(flat)


def test_traced_solve_records_targets(hwmod):
    w = inputs.tiny()
    ctx = hwmod.Context(0)
    L = ctx.setup_basis(w.geom, w.etas)
    ctx.build_potential(w.atoms)
    r = ctx.solve_traced(0, w.n_eig, 12, [1, 3], tol=1e-8, maxit=300)
    assert r["converged"]
    plain = ctx.solve_eigs([0], w.n_eig, block=12, tol=1e-8, maxit=300)
    assert np.abs(plain["evals"][0] - r["evals"]).max() < 1e-9
    R, E = r["R"], r["E"]
    assert torch.isfinite(R).all() and torch.isfinite(E).all()
    # every recorded residual norm matches its block column
    np.testing.assert_allclose(torch.linalg.norm(R, dim=2).cpu().numpy(), r["res"], rtol=1e-10)
    # corrections are nonzero where the residual is
    assert (torch.linalg.norm(E, dim=2)[0, :w.n_eig] > 0).all()
