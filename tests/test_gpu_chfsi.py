"""GPU parity of the alternative eigensolver, Chebyshev-filtered subspace iteration
(hw_set_option(HW_OPT_EIGENSOLVER, 1)), against the oracle's dense eigenvalues
(tests/golden/, written by tests/golden/make_golden.py from the oracle alone).

Tolerances as for LOBPCG: 1e-8 Ha in FP64, 1e-6 Ha in the mixed form; every reported residual
at most the requested 1e-6.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2210_12252_gb300 import inputs

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    return np.loadtxt(os.path.join(GOLD, name))


@pytest.fixture(scope="module")
def hwmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_12252_gb300 import build
    build.build()
    from paper_2210_12252_gb300 import helicwave
    return helicwave


def make_ctx(hwmod, w, degree=None):
    ctx = hwmod.Context(0)
    L = ctx.setup_basis(w.geom, w.etas, w.nus)
    ctx.build_potential(w.atoms)
    ctx.set_option(hwmod.HW_OPT_EIGENSOLVER, 1)
    if degree is not None:
        ctx.set_option(hwmod.HW_OPT_CHEB_DEGREE, degree)
    return ctx, L


@pytest.mark.parametrize("degree", [4, 16])
def test_chfsi_tiny_fp64_matches_dense_oracle(hwmod, degree):
    w = inputs.tiny()
    ctx, L = make_ctx(hwmod, w, degree)
    r = ctx.solve_eigs([0], w.n_eig, tol=1e-6, maxit=300, vectors=True)
    assert r["converged"]
    assert np.abs(r["evals"][0] - golden("tiny_eigs.txt")[: w.n_eig]).max() < 1e-8
    assert r["resid"].max() <= 1e-6
    X = r["evecs"][0]
    G = (X.conj() @ X.T).cpu().numpy()
    assert np.abs(G - np.eye(w.n_eig)).max() < 1e-10
    HX = ctx.apply_H(0, X.contiguous())
    res = torch.linalg.norm(HX - torch.from_numpy(r["evals"][0]).cuda()[:, None] * X, dim=1)
    assert res.max().item() <= 1.01e-6


@pytest.mark.parametrize("lock,adapt", [(0, 0), (0, 1), (1, 0)])
def test_chfsi_tube_fp64_option_paths(hwmod, lock, adapt):
    """The non-default paths: every column filtered every cycle and/or the full degree in every
    FP64 cycle reach the same eigenvalues."""
    w = inputs.tube()
    ctx, L = make_ctx(hwmod, w)
    ctx.set_option(hwmod.HW_OPT_CHEB_LOCK, lock)
    ctx.set_option(hwmod.HW_OPT_CHEB_ADAPT, adapt)
    r = ctx.solve_eigs([0], 32, tol=1e-6, maxit=100)
    assert r["converged"]
    assert np.abs(r["evals"][0] - golden("tube_eigs.txt")[:32]).max() < 1e-8
    assert r["resid"].max() <= 1e-6


def test_chfsi_tiny_cyclic_nu_fp64(hwmod):
    """nu != 0 points (the spectral bound carries the 1/r^2 term) in one batched solve."""
    w = inputs.tiny_cyclic()
    ctx, L = make_ctx(hwmod, w)
    r = ctx.solve_eigs([0, 1, 2], w.n_eig, tol=1e-6, maxit=300)
    assert r["converged"]
    for k in range(3):
        assert np.abs(r["evals"][k] - golden(f"tiny_c3_k{k}_eigs.txt")[: w.n_eig]).max() < 1e-8, k


@pytest.mark.parametrize("prec,tol_ev", [("fp64", 1e-8), ("mixed", 1e-6)])
def test_chfsi_tube_matches_dense_oracle(hwmod, prec, tol_ev):
    w = inputs.tube()
    ctx, L = make_ctx(hwmod, w)
    r = ctx.solve_eigs([0], w.n_eig, tol=1e-6, maxit=100, prec=prec)
    assert r["converged"]
    assert np.abs(r["evals"][0] - golden("tube_eigs.txt")[: w.n_eig]).max() < tol_ev
    assert r["resid"].max() <= 1e-6


def test_chfsi_batched_uneven_cyclic_mixed(hwmod):
    """Three (eta, nu) points of the Ncyc = 3 tube with uneven bases in one lockstep solve."""
    w = inputs.tube_cyclic()
    ctx, L = make_ctx(hwmod, w)
    r = ctx.solve_eigs([0, 1, 2], w.n_eig, tol=1e-6, maxit=100, prec="mixed")
    assert r["converged"]
    for k in range(3):
        assert np.abs(r["evals"][k] - golden(f"tube_c3_k{k}_eigs.txt")[: w.n_eig]).max() < 1e-6, k
    assert r["resid"].max() <= 1e-6


def test_chfsi_tube_fp64_maximum_block(hwmod):
    """The largest block the solvers take (112 columns) with the Chebyshev solver in FP64."""
    w = inputs.tube()
    ctx, L = make_ctx(hwmod, w)
    r = ctx.solve_eigs([0], 64, block=112, tol=1e-6, maxit=100)
    assert r["converged"]
    assert np.abs(r["evals"][0] - golden("tube_eigs.txt")[:64]).max() < 1e-8


@pytest.mark.parametrize("solver", [0, 1])
def test_solve_rejects_bad_arguments(hwmod, solver):
    w = inputs.tiny()
    ctx = hwmod.Context(0)
    ctx.setup_basis(w.geom, w.etas)
    ctx.build_potential(w.atoms)
    ctx.set_option(hwmod.HW_OPT_EIGENSOLVER, solver)
    for kw in [dict(kidx=[1], n_eig=8), dict(kidx=[0], n_eig=0), dict(kidx=[0], n_eig=8, block=6),
               dict(kidx=[0], n_eig=8, block=113), dict(kidx=[0], n_eig=8, block=99),
               dict(kidx=[0], n_eig=8, tol=0.0)]:
        args = dict(block=0, tol=1e-6)
        args.update(kw)
        kidx, n_eig = args.pop("kidx"), args.pop("n_eig")
        with pytest.raises(hwmod.HwError) as e:
            ctx.solve_eigs(kidx, n_eig, **args)
        assert e.value.status == hwmod.HW_EINVAL, kw


def test_chfsi_tube_mixed_overlap_bit_identical(hwmod):
    """The chosen form with and without overlapped launches of the FP32 H X chain (the filter's
    recurrence steps fused into the forward radial kernel): the same start block gives the same
    eigenvalues bit for bit and the same number of cycles + iterations."""
    w = inputs.tube()
    res = {}
    for ov in (1, 0):
        ctx, L = make_ctx(hwmod, w)
        ctx.set_option(hwmod.HW_OPT_OVERLAP_LAUNCH, ov)
        X0 = torch.from_numpy(np.ascontiguousarray(inputs.random_block(int(L[0]), 76, 1234).T)).cuda()
        r = ctx.solve_eigs([0], w.n_eig, block=76, tol=1e-6, maxit=100, prec="mixed", X0=[X0])
        assert r["converged"]
        res[ov] = r
        ctx.close()
    assert np.array_equal(res[1]["evals"][0], res[0]["evals"][0])
    assert np.array_equal(np.asarray(res[1]["iters"]), np.asarray(res[0]["iters"]))
    assert np.abs(res[1]["evals"][0] - golden("tube_eigs.txt")[: w.n_eig]).max() < 1e-6


@pytest.mark.parametrize("block", [80, 95])
def test_chfsi_tube_mixed_wide_block_takes_householder_route(hwmod, block):
    """Blocks whose 3 nb Rayleigh-Ritz size (LOBPCG's [X W P]) does not fit one CTA's shared
    memory (nb > 78) still take the Householder route for the smaller sizes (the filter's nb, the
    end phase's [X W]); they once fell to the Jacobi solver for every step (2-3x slower).  The
    phase profile records the reduction's launches only on the Householder route."""
    w = inputs.tube()
    ctx, L = make_ctx(hwmod, w, degree=28)
    X0 = torch.from_numpy(np.ascontiguousarray(inputs.random_block(int(L[0]), block, 1234).T)).cuda()
    ctx.profile(True)
    r = ctx.solve_eigs([0], w.n_eig, block=block, tol=1e-6, maxit=100, prec="mixed", X0=[X0])
    prof = ctx.profile_read()
    ctx.profile(False)
    assert r["converged"]
    assert prof["tridiag"][1] > 0
    assert np.abs(r["evals"][0] - golden("tube_eigs.txt")[: w.n_eig]).max() < 1e-6
    ctx.close()
