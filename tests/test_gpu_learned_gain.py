"""What the trained preconditioner network gains over the method without it.

Uses the committed weights (paper_2210_12252_gb300/precond_weights.npy, trained on the GPU by
train_precond.py with the library's own kernels on 256 seeded potentials of the random family).
On held-out members of that family the learned scaling must need fewer LOBPCG iterations than
the TPA diagonal for the same residual bar and give the same eigenvalues; on the tube workload
its eigenvalues must stay within the mixed-precision bar (1e-6 Ha) of the dense oracle.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2210_12252_gb300 import inputs

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_12252_gb300 import build, helicwave, train_precond
    build.build()
    c = helicwave.Context(0)
    c.setup_basis(inputs.GEOM_TUBE, [0.0])
    c.set_mlp(train_precond.load_weights())
    return c


@pytest.mark.parametrize("index", [256, 290, 319])
def test_learned_needs_fewer_iterations_on_heldout_potentials(ctx, index):
    w = inputs.tube_family(index)
    ctx.build_potential(w.atoms)
    r_tpa = ctx.solve_eigs([0], w.n_eig, tol=1e-6, maxit=600, prec="mixed", precond="tpa")
    r_ml = ctx.solve_eigs([0], w.n_eig, tol=1e-6, maxit=600, prec="mixed", precond="learned")
    assert r_tpa["converged"] and r_ml["converged"]
    assert r_ml["iters"][0] < r_tpa["iters"][0], (r_ml["iters"], r_tpa["iters"])
    assert np.abs(r_ml["evals"] - r_tpa["evals"]).max() < 1e-7
    assert r_ml["resid"].max() <= 1e-6


def test_learned_form_matches_oracle_on_tube(ctx):
    w = inputs.tube()
    ctx.build_potential(w.atoms)
    r = ctx.solve_eigs([0], w.n_eig, tol=1e-6, maxit=600, prec="mixed", precond="learned")
    assert r["converged"]
    ref = np.loadtxt(os.path.join(GOLD, "tube_eigs.txt"))[: w.n_eig]
    assert np.abs(r["evals"][0] - ref).max() < 1e-6
