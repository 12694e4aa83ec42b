"""Pins of the oracle's preconditioner network: gradients against central finite differences of
the loss, the zero-last-layer start equal to the TPA diagonal, BF16 rounding against torch's
bfloat16 conversion, and the potential diagonal against the diagonal of the dense Hamiltonian."""
import numpy as np
import pytest

from oracle import basis as B
from oracle import eigensolver as E
from oracle import hamiltonian as Hm
from oracle import mlp as Mo
from oracle import potential as P
from paper_2210_12252_gb300 import inputs


def tiny_kp():
    w = inputs.tiny()
    g = w.geom
    b = B.Basis(g.R, g.tau, g.alpha, g.Nr, g.Nth1, g.Nth2)
    V = P.gaussian_wells(b, w.atoms)
    return B.KPoint(b, 0.1, 0.0, 12.0), V


def test_potential_diagonal_is_the_diagonal_of_the_dense_hamiltonian():
    kp, V = tiny_kp()
    H = Hm.dense_H(kp, V)
    vd = Mo.potential_diagonal(kp, V)
    np.testing.assert_allclose(vd, np.real(np.diag(H)) - kp.ke, rtol=1e-12, atol=1e-12)


def test_gradients_match_finite_differences():
    kp, V = tiny_kp()
    rng = np.random.default_rng(4)
    params = Mo.init_params(1)
    params[4] = rng.standard_normal(Mo.HIDDEN) * 0.1      # nonzero last layer
    params[5] = np.array([0.05])
    vd = Mo.potential_diagonal(kp, V)
    X = Mo.features(kp, vd, theta=-1.3)
    r = rng.standard_normal(kp.L) + 1j * rng.standard_normal(kp.L)
    e = rng.standard_normal(kp.L) + 1j * rng.standard_normal(kp.L)
    tpa = Mo.tpa_factor(kp.ke, r)
    loss, grads = Mo.column_loss_and_grad(params, X, tpa, r, e)
    h = 1e-6
    for pi, (p, g) in enumerate(zip(params, grads)):
        flat = p.reshape(-1)
        gflat = np.asarray(g).reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = Mo.column_loss_and_grad(params, X, tpa, r, e)
            flat[idx] = old - h
            lm, _ = Mo.column_loss_and_grad(params, X, tpa, r, e)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gflat[idx]) < 1e-6 * max(1.0, abs(fd)), (pi, idx, fd, gflat[idx])


def test_zero_last_layer_reproduces_tpa():
    kp, V = tiny_kp()
    params = Mo.init_params(2)
    X = Mo.features(kp, Mo.potential_diagonal(kp, V), 0.5)
    o, _ = Mo.forward(params, X)
    assert np.all(o == 0.0)
    r = np.random.default_rng(1).standard_normal((kp.L, 1)) + 0j
    np.testing.assert_allclose(Mo.tpa_factor(kp.ke, r[:, 0]) * r[:, 0], E.tpa(kp.ke, r)[:, 0],
                               rtol=1e-14)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).standard_normal(1000) * 10
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(Mo.bf16_round(x), ref)
