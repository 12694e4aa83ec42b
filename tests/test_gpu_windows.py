"""Windowed solves (more eigenpairs than one block holds): consecutive windows of eigenpairs,
each a block solve in the orthogonal complement of the eigenvectors the earlier windows
converged (hw_solve_eigs, HW_OPT_WINDOW).

The tube cases compare every eigenvalue with the oracle's dense diagonalisation
(tests/golden/, written by tests/golden/make_golden.py from the oracle alone): 1e-8 Ha in FP64,
1e-6 Ha in the mixed form; the vectors of all windows together must be orthonormal to 1e-8.
The nanowire case (the full-size basis, L = 40,527, 400 eigenpairs) has no dense oracle: its
eigenpairs are checked through the oracle's own H X on sampled columns (residual at most the
requested 1e-6 with a rounding margin), for ascending order and for orthonormality.
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


def make_ctx(hwmod, w):
    ctx = hwmod.Context(0)
    L = ctx.setup_basis(w.geom, w.etas, w.nus)
    ctx.build_potential(w.atoms)
    ctx.set_option(hwmod.HW_OPT_EIGENSOLVER, 1)
    return ctx, L


@pytest.fixture(scope="module")
def hwmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_12252_gb300 import build
    build.build()
    from paper_2210_12252_gb300 import helicwave
    return helicwave


def gram_err(X):
    G = (X.conj() @ X.T).cpu().numpy()
    return np.abs(G - np.eye(G.shape[0])).max()


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("prec,tol_ev", [("fp64", 1e-8), ("mixed", 1e-6)])
def test_tube_120_eigenpairs_in_two_windows(hwmod, solver, prec, tol_ev):
    """120 > 80 eigenpairs: the default window splits them into two windows of 60."""
    w = inputs.tube()
    ctx, L = make_ctx(hwmod, w)
    ctx.set_option(hwmod.HW_OPT_EIGENSOLVER, solver)
    r = ctx.solve_eigs([0], 120, tol=1e-6, maxit=200, prec=prec)
    assert r["converged"]
    assert np.abs(r["evals"][0] - golden("tube_eigs.txt")[:120]).max() < tol_ev
    assert r["resid"].max() <= 1e-6


def test_tube_windows_of_24_vectors_orthonormal(hwmod):
    """64 eigenpairs in three windows (22, 22, 20) in the chosen form: eigenvalues, the
    orthonormality of all 64 vectors across the windows, and their residuals."""
    w = inputs.tube()
    ctx, L = make_ctx(hwmod, w)
    ctx.set_option(hwmod.HW_OPT_WINDOW, 24)
    r = ctx.solve_eigs([0], 64, tol=1e-6, maxit=200, prec="mixed", vectors=True)
    assert r["converged"]
    assert np.abs(r["evals"][0] - golden("tube_eigs.txt")[:64]).max() < 1e-6
    X = r["evecs"][0]
    assert gram_err(X) < 1e-8
    HX = ctx.apply_H(0, X.contiguous())
    res = torch.linalg.norm(HX - torch.from_numpy(r["evals"][0]).cuda()[:, None] * X, dim=1)
    assert res.max().item() <= 1.01e-6


def test_batched_cyclic_windows_uneven_bases(hwmod):
    """Three (eta, nu) points of the Ncyc = 3 tube (uneven bases) in lockstep windows of 11, 11
    and 10 eigenpairs."""
    w = inputs.tube_cyclic()
    ctx, L = make_ctx(hwmod, w)
    ctx.set_option(hwmod.HW_OPT_WINDOW, 12)
    r = ctx.solve_eigs([0, 1, 2], w.n_eig, tol=1e-6, maxit=200, prec="mixed", vectors=True)
    assert r["converged"]
    for k in range(3):
        assert np.abs(r["evals"][k] - golden(f"tube_c3_k{k}_eigs.txt")[: w.n_eig]).max() < 1e-6, k
        assert gram_err(r["evecs"][k][:, : L[k]]) < 1e-8, k
    assert r["resid"].max() <= 1e-6


def test_windowed_solve_rejects_a_start_block(hwmod):
    w = inputs.tube()
    ctx, L = make_ctx(hwmod, w)
    X0 = [torch.zeros((112, int(L[0])), dtype=torch.complex128, device="cuda")]
    with pytest.raises(hwmod.HwError) as e:
        ctx.solve_eigs([0], 120, tol=1e-6, X0=X0)
    assert e.value.status == hwmod.HW_EINVAL


def test_wire_400_eigenpairs_chosen_form(hwmod):
    """The nanowire configuration's eigenproblem size at one k-point: 400 eigenpairs in five
    windows of 80 (blocks of 112) on the full-size basis, chosen form (mixed precision,
    Chebyshev filtering then the LOBPCG end phase).  The potential is the workload's first 20
    wells (as in tests/test_gpu_wire.py), so that the oracle builds V in seconds."""
    from oracle import basis as B
    from oracle import hamiltonian as Hm
    from oracle import potential as P
    w = inputs.wire(nk=1)
    g = w.geom
    atoms = w.atoms[:20]
    ctx = hwmod.Context(0)
    L = ctx.setup_basis(g, w.etas[:1])
    ctx.build_potential(atoms)
    ctx.set_option(hwmod.HW_OPT_EIGENSOLVER, 1)
    r = ctx.solve_eigs([0], 400, tol=1e-6, maxit=200, prec="mixed", vectors=True)
    assert r["converged"]
    ev = r["evals"][0]
    assert r["resid"].max() <= 1e-6
    assert np.all(np.diff(ev) > -1e-9)
    X = r["evecs"][0]
    assert gram_err(X) < 1e-8
    # sampled eigenpairs against the oracle's H X (one column per window and the last)
    b = B.Basis(g.R, g.tau, g.alpha, g.Nr, g.Nth1, g.Nth2, g.ncyc, g.oversample)
    kp = B.KPoint(b, w.etas[0], 0.0, g.ecut)
    assert kp.L == L[0]
    V = P.gaussian_wells(b, atoms)
    cols = [0, 150, 250, 399]
    Xs = X[cols].cpu().numpy().T
    HXs = Hm.apply_H(kp, V, Xs)
    res = np.linalg.norm(HXs - ev[cols][None, :] * Xs, axis=0)
    assert res.max() <= 1.05e-6
