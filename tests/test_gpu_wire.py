"""Parity at the full nanowire-like size (R=20, tau=8, alpha=0.02, N_r=192, 192 x 96 angular grid,
40 Ha cutoff: L = 40,527 at the first seeded eta): sampled columns of H X (FP64 and mixed), the
mixed electron density of two states, and the Cartesian gradient of one column, each against
the CPU oracle on the same seeded inputs.

The potential is the workload's Gaussian wells restricted to its first 20 (of 300) atoms, so
that the oracle builds it in seconds; the basis, grids and launch shapes are the full-size
ones (the H X kernels do not depend on how many wells make up V).  Tolerances as on the small
cases: H X 1e-10 (FP64) / 2e-6 (mixed) relative per column; density 2e-6 of max rho (mixed);
gradient 1e-10 (FP64).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import basis as B
from oracle import density as D
from oracle import gradient as Gr
from oracle import hamiltonian as Hm
from oracle import potential as P
from paper_2210_12252_gb300 import inputs
from _parity import assert_entrywise

pytestmark = pytest.mark.gpu
N_ATOMS = 20


@pytest.fixture(scope="module")
def hwmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_12252_gb300 import build
    build.build()
    from paper_2210_12252_gb300 import helicwave
    return helicwave


@pytest.fixture(scope="module")
def wire(hwmod):
    w = inputs.wire(nk=1)
    g = w.geom
    atoms = w.atoms[:N_ATOMS]
    ctx = hwmod.Context(0)
    L = ctx.setup_basis(g, w.etas[:1])
    ctx.build_potential(atoms)
    b = B.Basis(g.R, g.tau, g.alpha, g.Nr, g.Nth1, g.Nth2, g.ncyc, g.oversample)
    kp = B.KPoint(b, w.etas[0], 0.0, g.ecut)
    assert L[0] == kp.L
    V = P.gaussian_wells(b, atoms)
    return ctx, kp, V


def to_dev(X):
    return torch.from_numpy(np.ascontiguousarray(X.T)).cuda()


def rel_err(Y, Yref):
    return (np.linalg.norm(Y - Yref, axis=0) / np.linalg.norm(Yref, axis=0)).max()


def test_wire_apply_H_sampled_columns(wire):
    ctx, kp, V = wire
    X = inputs.random_block(kp.L, 2, 91)
    Yref = Hm.apply_H(kp, V, X)
    Xd = to_dev(X)
    Y64 = ctx.apply_H(0, Xd).cpu().numpy().T
    assert rel_err(Y64, Yref) < 1e-10
    assert_entrywise(Y64, Yref, 1e-10, 1e-13, "wire fp64")
    Y32 = ctx.apply_H(0, Xd, prec="mixed").cpu().numpy().T
    e = rel_err(Y32, Yref)
    assert 1e-12 < e < 2e-6
    assert_entrywise(Y32, Yref, 2e-6, 2e-7, "wire mixed")


def test_wire_density_mixed_two_states(wire):
    ctx, kp, V = wire
    g = np.random.default_rng(92)
    Q, _ = np.linalg.qr(g.standard_normal((kp.L, 2)) + 1j * g.standard_normal((kp.L, 2)))
    occ = np.array([[1.0, 0.5]])
    rho = ctx.density([0], [to_dev(Q)], occ, [1.0], prec="mixed").cpu().numpy()
    ref = D.density([kp], [Q], occ, [1.0])
    assert np.abs(rho - ref).max() < 2e-6 * np.abs(ref).max()
    assert_entrywise(rho.ravel(), ref.ravel(), 2e-6, 2e-7, "wire density mixed")


def test_wire_gradient_fp64_one_column(wire):
    ctx, kp, V = wire
    X = inputs.random_block(kp.L, 1, 93)
    Dd = ctx.gradient(0, to_dev(X)).cpu().numpy()
    ref = Gr.gradient(kp, X[:, 0])
    for comp in range(3):
        assert np.abs(Dd[0, comp] - ref[comp]).max() < 1e-10 * np.abs(ref[comp]).max()
        assert_entrywise(Dd[0, comp].ravel(), ref[comp].ravel(), 1e-10, 1e-13, f"wire gradient {comp}")


def test_wire_potential_all_300_wells_at_sampled_points(hwmod):
    """The library's host-built potential of the nanowire workload with all 300 wells, against
    the oracle's image sum at 20,000 seeded grid points (the oracle's full-grid build of 300
    wells takes minutes; the image sum is the same at each point)."""
    w = inputs.wire(nk=1)
    g = w.geom
    assert len(w.atoms) == 300
    ctx = hwmod.Context(0)
    ctx.setup_basis(g, w.etas[:1])
    V = ctx.build_potential(w.atoms).reshape(g.Nth1, g.Nth2, g.Nr)
    b = B.Basis(g.R, g.tau, g.alpha, g.Nr, g.Nth1, g.Nth2, g.ncyc, g.oversample)
    rng = np.random.default_rng(301)
    i, j, p = (rng.integers(0, n, 20000) for n in (g.Nth1, g.Nth2, g.Nr))
    ref = P.gaussian_wells_at(b, w.atoms, i, j, p)
    assert np.abs(ref).max() > 1.0                    # the sample sees the wells
    assert_entrywise(V[i, j, p], ref, 1e-12, 1e-13, "300-well potential")
    ctx.close()
