"""GPU parity with a cyclic symmetry (Ncyc = 3) and cyclic wavenumbers nu != 0: H X with the
1/r^2 terms of the I_n loop of Algorithm 5 (through the C ABI) against the CPU oracle, and the
eigensolver against the oracle's dense eigenvalues (tests/golden/, written by
tests/golden/make_golden.py from the oracle alone).

Tolerances as for nu = 0: H X to 1e-10 relative (FP64) and 2e-6 (mixed) per column, and every
entry within tol |Y_ij| + floor max_i |Y_ij| (floors 1e-13 / 2e-7, as in test_gpu_hx.py);
eigenvalues to 1e-8 Ha (FP64) and 1e-6 Ha (mixed).
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import basis as B
from oracle import hamiltonian as Hm
from oracle import potential as P
from paper_2210_12252_gb300 import inputs
from _parity import assert_entrywise

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 2e-6
FP64_FLOOR = 1e-13
MIXED_FLOOR = 2e-7
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


def to_dev(X, ld=None):
    L, ns = X.shape
    ld = ld or L
    T = torch.zeros((ns, ld), dtype=torch.complex128)
    T[:, :L] = torch.from_numpy(np.ascontiguousarray(X.T))
    return T.cuda()


def from_dev(T, L):
    return T[:, :L].cpu().numpy().T


def rel_err(Y, Yref):
    return (np.linalg.norm(Y - Yref, axis=0) / np.linalg.norm(Yref, axis=0)).max()


class Case:
    def __init__(self, hwmod, w):
        g = w.geom
        self.w = w
        self.ctx = hwmod.Context(0)
        self.L = self.ctx.setup_basis(g, w.etas, w.nus)
        self.ctx.build_potential(w.atoms)
        self.b = B.Basis(g.R, g.tau, g.alpha, g.Nr, g.Nth1, g.Nth2, g.ncyc, g.oversample)
        self.V = P.gaussian_wells(self.b, w.atoms)
        self.kps = [B.KPoint(self.b, e, nu, g.ecut) for e, nu in zip(w.etas, w.nus)]


@pytest.fixture(scope="module")
def tiny(hwmod):
    return Case(hwmod, inputs.tiny_cyclic())


@pytest.fixture(scope="module")
def tube(hwmod):
    return Case(hwmod, inputs.tube_cyclic())


@pytest.mark.parametrize("ns", [1, 7])
def test_apply_H_fp64_tiny_each_nu(tiny, ns):
    for k, kp in enumerate(tiny.kps):
        assert tiny.L[k] == kp.L
        X = inputs.random_block(kp.L, ns, 40 + k)
        Yref = Hm.apply_H(kp, tiny.V, X)
        Y = from_dev(tiny.ctx.apply_H(k, to_dev(X)), kp.L)
        assert rel_err(Y, Yref) < FP64_TOL, (k, kp.nu)
        assert_entrywise(Y, Yref, FP64_TOL, FP64_FLOOR, f"tiny k{k} nu={kp.nu}")


def test_apply_H_mixed_tiny_nu(tiny):
    kp = tiny.kps[1]
    X = inputs.random_block(kp.L, 4, 51)
    Yref = Hm.apply_H(kp, tiny.V, X)
    Y = from_dev(tiny.ctx.apply_H(1, to_dev(X), prec="mixed"), kp.L)
    e = rel_err(Y, Yref)
    assert 1e-12 < e < MIXED_TOL
    assert_entrywise(Y, Yref, MIXED_TOL, MIXED_FLOOR, "tiny mixed nu")


def test_apply_H_is_hermitian_with_nu(tiny):
    kp = tiny.kps[0]
    X = inputs.random_block(kp.L, 6, 52)
    Y = from_dev(tiny.ctx.apply_H(0, to_dev(X)), kp.L)
    G = X.conj().T @ Y
    assert np.abs(G - G.conj().T).max() < 1e-12 * np.abs(G).max()


def test_apply_H_batched_tube_cyclic_ragged(tube):
    """The three (eta, nu) points of the Ncyc = 3 tube in one batched launch (uneven L, padded
    leading dimension), sampled columns against the oracle's Algorithm 5."""
    ns = 2
    Lmax = int(max(tube.L))
    Xs, Ys, refs = [], [], []
    for k, kp in enumerate(tube.kps):
        assert tube.L[k] == kp.L
        X = inputs.random_block(kp.L, ns, 60 + k)
        Xs.append(to_dev(X, ld=Lmax + 5))
        Ys.append(torch.zeros_like(Xs[-1]))
        refs.append(Hm.apply_H(kp, tube.V, X))
    tube.ctx.apply_H_batched([0, 1, 2], Xs, Ys)
    for k, kp in enumerate(tube.kps):
        assert rel_err(from_dev(Ys[k], kp.L), refs[k]) < FP64_TOL, k
        assert_entrywise(from_dev(Ys[k], kp.L), refs[k], FP64_TOL, FP64_FLOOR, f"tube c3 k{k} fp64")
    tube.ctx.apply_H_batched([0, 1, 2], Xs, Ys, prec="mixed")
    for k, kp in enumerate(tube.kps):
        assert rel_err(from_dev(Ys[k], kp.L), refs[k]) < MIXED_TOL, k
        assert_entrywise(from_dev(Ys[k], kp.L), refs[k], MIXED_TOL, MIXED_FLOOR, f"tube c3 k{k} mixed")


def test_solve_tiny_cyclic_fp64_matches_dense_oracle(tiny, hwmod):
    w = tiny.w
    r = tiny.ctx.solve_eigs([0, 1, 2], w.n_eig, tol=1e-6, maxit=400)
    assert r["converged"]
    for k in range(3):
        ref = golden(f"tiny_c3_k{k}_eigs.txt")[: w.n_eig]
        assert np.abs(r["evals"][k] - ref).max() < 1e-8, k
    assert r["resid"].max() <= 1e-6


def test_solve_tube_cyclic_mixed_matches_dense_oracle(tube):
    w = tube.w
    r = tube.ctx.solve_eigs([0, 1, 2], w.n_eig, tol=1e-6, maxit=400, prec="mixed")
    assert r["converged"]
    for k in range(3):
        ref = golden(f"tube_c3_k{k}_eigs.txt")[: w.n_eig]
        assert np.abs(r["evals"][k] - ref).max() < 1e-6, k
    assert r["resid"].max() <= 1e-6
