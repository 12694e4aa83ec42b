"""Pins of the density oracle (oracle/density.py) against facts outside it.

1. One basis function F_{m,n,k} as the only state: |F|^2 = xi_{n,k}(r)^2 is independent of the
   angles, so rho = 2 w s xi^2 on every angular node; xi from scipy's Bessel J and the zeros
   of J_n found here by scipy's brentq (not the oracle's tables).
2. Orthonormal states in the basis: the forward-transform quadrature of rho is the electron
   count 2 sum_b w_b sum_j s_j up to the radial quadrature error.
3. The fast path (Algorithms 1-2) equals the direct sum of eq. Naive_Inverse_Transform.
"""
import math

import numpy as np
import pytest
from scipy import optimize, special

from oracle import basis as B
from oracle import density as D


@pytest.fixture(scope="module")
def small():
    b = B.Basis(R=6.0, tau=3.0, alpha=0.1, Nr=24, Nth1=16, Nth2=16)
    kp = B.KPoint(b, 0.0, 0.0, None)
    return b, kp


def jn_zero(n, k):
    """k-th (0-based) positive zero of J_n by bracketing on a fine grid + brentq."""
    x = np.linspace(1e-6, 80.0, 80001)
    f = special.jv(n, x)
    roots = [optimize.brentq(lambda t: special.jv(n, t), x[i], x[i + 1])
             for i in np.nonzero(np.sign(f[:-1]) * np.sign(f[1:]) < 0)[0]]
    return roots[k]


@pytest.mark.parametrize("m,n,k", [(0, 0, 0), (2, -1, 1), (-3, 2, 4)])
def test_single_basis_function(small, m, n, k):
    b, kp = small
    x = np.zeros(kp.L, dtype=complex)
    i = np.nonzero((kp.m == m) & (kp.n == n) & (kp.k == k))[0][0]
    x[i] = 1.0
    rho = D.density([kp], [x[:, None]], [np.array([0.75])], [0.5])
    bz = jn_zero(abs(n), k)
    c = math.sqrt(1.0 / (math.pi * b.tau)) / (b.R * special.jv(abs(n) + 1, bz))
    xi = c * special.jv(abs(n), bz * b.r / b.R)
    expect = 2 * 0.5 * 0.75 * xi ** 2
    np.testing.assert_allclose(rho, np.broadcast_to(expect, rho.shape), rtol=1e-10, atol=1e-14)


def test_charge_of_orthonormal_states(small):
    b, kp = small
    g = np.random.default_rng(3)
    Q, _ = np.linalg.qr(g.standard_normal((kp.L, 5)) + 1j * g.standard_normal((kp.L, 5)))
    occ = np.array([1.0, 1.0, 0.5, 0.25, 0.0])
    rho = D.density([kp, kp], [Q, Q[:, ::-1]], [occ, occ], [0.5, 0.5])
    assert abs(D.charge(b, rho) - 2 * occ.sum()) < 1e-9
    assert rho.min() >= 0.0


def test_fast_equals_naive(small):
    b, kp = small
    g = np.random.default_rng(4)
    X = g.standard_normal((kp.L, 2)) + 1j * g.standard_normal((kp.L, 2))
    r1 = D.density([kp], [X], [np.array([1.0, 0.3])], [1.0])
    r2 = D.density([kp], [X], [np.array([1.0, 0.3])], [1.0], naive=True)
    np.testing.assert_allclose(r1, r2, rtol=1e-12, atol=1e-12 * np.abs(r2).max())
